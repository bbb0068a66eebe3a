// dfv_gas.cuh -- the single-gas pieces shared by the stage kernels of 2-D
// (dfv_gasw.cuh) and 3-D (dfv_gas3.cuh) FP32 grids of one ideal or stiffened
// gas: the instance record of the 2-D kernel's work items, the van Leer
// slope, the gas closure and the HLLC flux.  The arithmetic per face and per
// cell is that of the general stage kernel (dfv_kernels.cuh) written for one
// gas: p = p_ref + Gamma (rho E - rho |u|^2/2), c^2 = (Gamma p + p - p_ref)/rho
// (Sec. 2.1.2).
#pragma once

#include "dfv_kernels.cuh"

namespace dfv {

// one grid served by the 2-D gas stage kernel (its work items: strips of
// columns x chunks of rows)
struct GasInst {
    int n0, n1;
    int strips, nitems;  // strips of 28 columns, work items (strips x chunks)
    long long off;       // element offset of the instance's planes
    long long pitch;     // elements between planes
    float idx, idy;      // 1/dx, 1/dy
    int wall_x0, wall_x1, wall_y0, wall_y1;   // reflective sides
    Ctl *ctl;
    int rows;            // rows per chunk
    int pad;
};

// ------------------------------------------------------------ arithmetic
//
// Every product below is either fused explicitly (fmaf) or rounded on its own
// (__fmul_rn), so that the compiler cannot contract it differently where the
// functions are inlined: a cell's result is then the same whichever code
// path (a chunk's first rows, its loop) computes it.
//
// Independent pairs of operations (the left and right states of a face, two
// components of a state) go to the packed FP32 units, two lanes of a float2
// per instruction.  Each lane rounds exactly as the scalar operation would
// (__fadd2_rn, __fmul2_rn, __ffma2_rn: per component __fadd_rn, __fmul_rn,
// __fmaf_rn), so the pairing changes the instruction count, not the result.

// approximate reciprocal: one hardware reciprocal (flush-to-zero)
__device__ __forceinline__ float gas_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 gas_f2(float x, float y) { return make_float2(x, y); }

// p - q per lane with one rounding (the negated product q * -1 is exact)
__device__ __forceinline__ float2 gas_sub2(float2 p, float2 q)
{
    return __ffma2_rn(q, make_float2(-1.f, -1.f), p);
}

// van Leer limited slope of a cell from its backward and forward differences
__device__ __forceinline__ float gas_vanleer(float a, float b)
{
    const float ab = __fmul_rn(a, b);
    return ab <= 0.f ? 0.f : __fmul_rn(ab + ab, gas_rcp(a + b));
}

// the same for two pairs of differences at once
__device__ __forceinline__ float2 gas_vanleer2(float2 a, float2 b)
{
    const float2 ab = __fmul2_rn(a, b);
    const float2 s = __fadd2_rn(a, b);
    const float2 q = __fmul2_rn(__fadd2_rn(ab, ab), gas_f2(gas_rcp(s.x), gas_rcp(s.y)));
    return gas_f2(ab.x <= 0.f ? 0.f : q.x, ab.y <= 0.f ? 0.f : q.y);
}

// Conserved (rho, rho u, rho v, rho E) -> primitive (rho, u, v, p) of the gas
// (a: any argument block with the gas constants Gam, invGam, pref0).
template <class A>
__device__ __forceinline__ void gas_prim(const A &a, float r, float mu, float mv, float E, float w[4])
{
    const float ir = gas_rcp(r);
    const float2 uv = __fmul2_rn(gas_f2(mu, mv), gas_f2(ir, ir));
    const float hr = __fmul_rn(0.5f, r);
    const float2 h = __fmul2_rn(gas_f2(hr, hr), uv);                   // (hr u, hr v)
    const float ke = fmaf(h.y, uv.y, __fmul_rn(h.x, uv.x));            // rho |u|^2 / 2
    w[0] = r;
    w[1] = uv.x;
    w[2] = uv.y;
    w[3] = fmaf(a.Gam, E - ke, a.pref0);
}

// HLLC flux of the gas across a face (Sec. 3.1: Toro's HLLC with Davis wave
// speeds), normal velocity un, tangential ut; F = (rho, normal momentum,
// tangential momentum, energy).  The left and right states' sound speeds,
// wave-speed bounds and contact-speed terms are formed pairwise.
template <class A>
__device__ __forceinline__ void gas_hllc(const A &a, float rL, float unL, float utL, float pL, float rR,
                                         float unR, float utR, float pR, float F[4])
{
    const float2 r2 = gas_f2(rL, rR), un2 = gas_f2(unL, unR), p2 = gas_f2(pL, pR);
    const float2 ir2 = gas_f2(gas_rcp(rL), gas_rcp(rR));
    const float2 cc = __fmul2_rn(__ffma2_rn(gas_f2(a.Gam, a.Gam), p2, gas_sub2(p2, gas_f2(a.pref0, a.pref0))), ir2);
    const float2 c2 = gas_f2(sqrtf(cc.x), sqrtf(cc.y));
    const float2 lo = gas_sub2(un2, c2), hi = __fadd2_rn(un2, c2);
    const float SL = fminf(lo.x, lo.y);
    const float SR = fmaxf(hi.x, hi.y);
    // contact speed, the numerator's products rounded one by one (a wall face
    // between mirror-image states gets S* = 0 exactly)
    const float2 d2 = gas_sub2(gas_f2(SL, SR), un2);                  // S_K - u_K
    const float2 mm = __fmul2_rn(__fmul2_rn(r2, un2), d2);
    const float num = __fadd_rn(__fadd_rn(pR - pL, mm.x), -mm.y);
    const float Ss = __fmul_rn(num, gas_rcp(fmaf(rL, d2.x, -__fmul_rn(rR, d2.y))));
    // regions: left of S_L, left star, right star, right of S_R
    const int region = SL >= 0.f ? 0 : (Ss >= 0.f ? 1 : (SR > 0.f ? 2 : 3));
    const bool left = region <= 1;
    const float r = left ? rL : rR, un = left ? unL : unR, ut = left ? utL : utR, p = left ? pL : pR;
    const float S = left ? SL : SR;
    const float hr = __fmul_rn(0.5f, r);
    const float2 h = __fmul2_rn(gas_f2(hr, hr), gas_f2(ut, un));       // (hr ut, hr un)
    const float E = fmaf(h.x, ut, fmaf(p - a.pref0, a.invGam, __fmul_rn(h.y, un)));
    const float m = __fmul_rn(r, un);
    // physical flux of the upwind side: (rho, normal momentum), (tangential momentum, energy)
    float2 Fa = gas_f2(m, fmaf(m, un, p));
    float2 Fb = __fmul2_rn(gas_f2(m, E + p), gas_f2(ut, un));
    const bool star = region == 1 || region == 2;
    if (star) {
        // star state U*_K = rho_K chi [1, S*, u_t, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))],
        // chi = (S_K - u_K)/(S_K - S*); with iD = 1/(S_K - S*) its energy is
        // chi E_K + (S* - u_K)(rho_K chi S* + p_K iD): one reciprocal
        const float2 dd = gas_sub2(gas_f2(S, S), gas_f2(Ss, un));   // (S_K - S*, S_K - u_K)
        const float iD = gas_rcp(dd.x);
        const float chi = __fmul_rn(dd.y, iD);
        const float rs = __fmul_rn(r, chi);
        const float Es = fmaf(chi, E, __fmul_rn(Ss - un, fmaf(rs, Ss, __fmul_rn(p, iD))));
        // F + S_K (U*_K - U_K)
        Fa = __ffma2_rn(gas_f2(S, S), gas_f2(rs - r, fmaf(rs, Ss, -m)), Fa);
        Fb = __ffma2_rn(gas_f2(S, S), gas_f2(fmaf(rs, ut, -__fmul_rn(r, ut)), Es - E), Fb);
    }
    F[0] = Fa.x;
    F[1] = Fa.y;
    F[2] = Fb.x;
    F[3] = Fb.y;
}

// Whether a 2-D grid can take the gas stage kernel: FP32, one ideal or
// stiffened gas, no solid, no periodic side, no HLLC-LM and a static body
// (the upwind r flux vanishes).
inline bool gas_eligible(int precision_fp32, int dim, int nmat, int solid, int mat_kind, const int periodic[3],
                         int hllc_lm, bool moving_body)
{
    return precision_fp32 && dim == 2 && nmat == 1 && solid == 0 && (mat_kind == 0 || mat_kind == 1) &&
           !periodic[0] && !periodic[1] && !hllc_lm && !moving_body;
}

}  // namespace dfv

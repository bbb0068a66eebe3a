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

// approximate reciprocal: one hardware reciprocal (flush-to-zero)
__device__ __forceinline__ float gas_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// van Leer limited slope of a cell from its backward and forward differences
__device__ __forceinline__ float gas_vanleer(float a, float b)
{
    const float ab = __fmul_rn(a, b);
    return ab <= 0.f ? 0.f : __fmul_rn(ab + ab, gas_rcp(a + b));
}

// Conserved (rho, rho u, rho v, rho E) -> primitive (rho, u, v, p) of the gas
// (a: any argument block with the gas constants Gam, invGam, pref0).
template <class A>
__device__ __forceinline__ void gas_prim(const A &a, float r, float mu, float mv, float E, float w[4])
{
    const float ir = gas_rcp(r);
    const float u = __fmul_rn(mu, ir), v = __fmul_rn(mv, ir);
    const float hr = __fmul_rn(0.5f, r);
    const float ke = fmaf(__fmul_rn(hr, v), v, __fmul_rn(__fmul_rn(hr, u), u));   // rho |u|^2 / 2
    w[0] = r;
    w[1] = u;
    w[2] = v;
    w[3] = fmaf(a.Gam, E - ke, a.pref0);
}

// HLLC flux of the gas across a face (Sec. 3.1: Toro's HLLC with Davis wave
// speeds), normal velocity un, tangential ut; F = (rho, normal momentum,
// tangential momentum, energy).
template <class A>
__device__ __forceinline__ void gas_hllc(const A &a, float rL, float unL, float utL, float pL, float rR,
                                         float unR, float utR, float pR, float F[4])
{
    const float irL = gas_rcp(rL), irR = gas_rcp(rR);
    const float cL = sqrtf(__fmul_rn(fmaf(a.Gam, pL, pL - a.pref0), irL));
    const float cR = sqrtf(__fmul_rn(fmaf(a.Gam, pR, pR - a.pref0), irR));
    const float SL = fminf(unL - cL, unR - cR);
    const float SR = fmaxf(unL + cL, unR + cR);
    // contact speed, the numerator's products rounded one by one (a wall face
    // between mirror-image states gets S* = 0 exactly)
    const float num = __fadd_rn(__fadd_rn(pR - pL, __fmul_rn(__fmul_rn(rL, unL), SL - unL)),
                                -__fmul_rn(__fmul_rn(rR, unR), SR - unR));
    const float Ss = __fmul_rn(num, gas_rcp(fmaf(rL, SL - unL, -__fmul_rn(rR, SR - unR))));
    // regions: left of S_L, left star, right star, right of S_R
    const int region = SL >= 0.f ? 0 : (Ss >= 0.f ? 1 : (SR > 0.f ? 2 : 3));
    const bool left = region <= 1;
    const float r = left ? rL : rR, un = left ? unL : unR, ut = left ? utL : utR, p = left ? pL : pR;
    const float S = left ? SL : SR;
    const float hr = __fmul_rn(0.5f, r);
    const float E = fmaf(__fmul_rn(hr, ut), ut, fmaf(p - a.pref0, a.invGam, __fmul_rn(__fmul_rn(hr, un), un)));
    const float m = __fmul_rn(r, un);
    // physical flux of the upwind side
    float Fr = m, Fn = fmaf(m, un, p), Ft = __fmul_rn(m, ut), FE = __fmul_rn(E + p, un);
    const bool star = region == 1 || region == 2;
    if (star) {
        // star state U*_K = rho_K chi [1, S*, u_t, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))],
        // chi = (S_K - u_K)/(S_K - S*); with iD = 1/(S_K - S*) its energy is
        // chi E_K + (S* - u_K)(rho_K chi S* + p_K iD): one reciprocal
        const float iD = gas_rcp(S - Ss);
        const float chi = __fmul_rn(S - un, iD);
        const float rs = __fmul_rn(r, chi);
        const float Es = fmaf(chi, E, __fmul_rn(Ss - un, fmaf(rs, Ss, __fmul_rn(p, iD))));
        Fr = fmaf(S, rs - r, Fr);
        Fn = fmaf(S, fmaf(rs, Ss, -m), Fn);
        Ft = fmaf(S, fmaf(rs, ut, -__fmul_rn(r, ut)), Ft);
        FE = fmaf(S, Es - E, FE);
    }
    F[0] = Fr;
    F[1] = Fn;
    F[2] = Ft;
    F[3] = FE;
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

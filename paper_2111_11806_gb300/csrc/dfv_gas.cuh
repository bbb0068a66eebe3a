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

// van Leer limited slope of a cell from its backward and forward differences
__device__ __forceinline__ float gas_vanleer(float a, float b)
{
    const float ab = a * b;
    return ab <= 0.f ? 0.f : __fdividef(2.f * ab, a + b);
}

// Conserved (rho, rho u, rho v, rho E) -> primitive (rho, u, v, p) of the gas
// (a: any argument block with the gas constants Gam, invGam, pref0).
template <class A>
__device__ __forceinline__ void gas_prim(const A &a, float r, float mu, float mv, float E, float w[4])
{
    const float ir = __fdividef(1.f, r);
    const float u = mu * ir, v = mv * ir;
    const float ke = 0.5f * r * u * u + 0.5f * r * v * v;
    w[0] = r;
    w[1] = u;
    w[2] = v;
    w[3] = a.pref0 + a.Gam * (E - ke);
}

// HLLC flux of the gas across a face (Sec. 3.1: Toro's HLLC with Davis wave
// speeds), normal velocity un, tangential ut; F = (rho, normal momentum,
// tangential momentum, energy).
template <class A>
__device__ __forceinline__ void gas_hllc(const A &a, float rL, float unL, float utL, float pL, float rR,
                                         float unR, float utR, float pR, float F[4])
{
    const float irL = __fdividef(1.f, rL), irR = __fdividef(1.f, rR);
    const float cL = sqrtf((a.Gam * pL + (pL - a.pref0)) * irL);
    const float cR = sqrtf((a.Gam * pR + (pR - a.pref0)) * irR);
    const float SL = fminf(unL - cL, unR - cR);
    const float SR = fmaxf(unL + cL, unR + cR);
    // contact speed, the numerator's products rounded one by one (a wall face
    // between mirror-image states gets S* = 0 exactly)
    const float num = __fadd_rn(__fadd_rn(pR - pL, __fmul_rn(__fmul_rn(rL, unL), SL - unL)),
                                -__fmul_rn(__fmul_rn(rR, unR), SR - unR));
    const float Ss = __fdividef(num, rL * (SL - unL) - rR * (SR - unR));
    // regions: left of S_L, left star, right star, right of S_R
    const int region = SL >= 0.f ? 0 : (Ss >= 0.f ? 1 : (SR > 0.f ? 2 : 3));
    const bool left = region <= 1;
    const float r = left ? rL : rR, un = left ? unL : unR, ut = left ? utL : utR, p = left ? pL : pR;
    const float S = left ? SL : SR;
    const float E = (p - a.pref0) * a.invGam + 0.5f * r * un * un + 0.5f * r * ut * ut;
    const float m = r * un;
    // physical flux of the upwind side
    float Fr = m, Fn = m * un + p, Ft = m * ut, FE = (E + p) * un;
    const bool star = region == 1 || region == 2;
    if (star) {
        // star state U*_K = rho_K chi [1, S*, u_t, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))],
        // chi = (S_K - u_K)/(S_K - S*); with iD = 1/(S_K - S*) its energy is
        // chi E_K + (S* - u_K)(rho_K chi S* + p_K iD): one reciprocal
        const float iD = __fdividef(1.f, S - Ss);
        const float chi = (S - un) * iD;
        const float rs = r * chi;
        const float Es = chi * E + (Ss - un) * (rs * Ss + p * iD);
        Fr += S * (rs - r);
        Fn += S * (rs * Ss - m);
        Ft += S * (rs * ut - r * ut);
        FE += S * (Es - E);
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

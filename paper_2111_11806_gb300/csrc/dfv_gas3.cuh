// dfv_gas3.cuh -- the SSP-RK3 stage (Sec. 3.1) of 3-D single-gas grids in
// FP32 (one ideal or stiffened gas, static body, transmissive or reflective
// sides): the form of the sphere workload.
//
// A CTA owns a 32 x 8 column of cells and marches through a chunk of planes
// in z.  A ring of three planes of primitives (z, z+1, z+2, each with its x
// and y halo of 2) sits in shared memory; per plane z:
//   1. plane z+2 is converted from the conserved values that arrived in the
//      shared fetch slot during the previous plane (one TMA tensor copy of
//      the plane's box, or per-thread asynchronous copies when rows are not
//      16-byte multiples); then plane z+3 is fetched into the slot, and the
//      cell's own values of plane z+1 are prefetched into L1;
//   2. slopes: every cell of plane z its van Leer slopes in x and y (face
//      values to shared memory, one warp the halo), every cell of plane z+1
//      its slope in z;
//   3. faces: every thread the HLLC fluxes of its cell's left x face, bottom
//      y face and top z face; the bottom z face and the top z-face value of
//      plane z were carried in shared memory from the previous plane;
//   4. update of plane z: divergence with a compensated (TwoSum) sum, rigid
//      mask, RK combination; in stage 3 the CFL maximum and the rigid box.
// Each primitive is converted once per chunk and each slope computed once;
// the arithmetic per face is that of the 2-D gas kernel (dfv_gas.cuh) with
// two tangential velocities.  Halo of 2: without a moving body the upwind r
// flux vanishes and r is not reconstructed (MUSCL only).
#pragma once

#include <cuda.h>

#include "dfv_gas.cuh"

namespace dfv {

// ------------------------------------------------------------ TMA, mbarrier

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase of parity `parity` to complete; false when the
// iteration limit ran out (the caller reports it and stops).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (int it = 0; it < (1 << 22); it++) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

struct Gas3T {
    static constexpr int TX = 32, TY = 8, H = 2;
    static constexpr int PX = TX + 2 * H, PY = TY + 2 * H;   // a plane with its x, y halo
    static constexpr int CELLS = TX * TY;
    static constexpr int THREADS = CELLS + 32;
    static constexpr int NCONV = TY * PX + 2 * H * TX;       // loaded cells of a plane (corners not)
    static constexpr int K = (NCONV + THREADS - 1) / THREADS; // loaded cells per thread
    static constexpr int RING = 3;
    static constexpr int NP = 6;                             // rho, rho u, rho v, rho w, rho E, r
    static constexpr int FXS = TX + 1, FYS = TY + 1;
    // planes per CTA (256^3 sphere, cell-updates/s at 16 / 24 / 32 / 48 / 64
    // planes: 8.59 / 8.64 / 8.40 / 8.52 / 8.04e9)
    static constexpr int ZCHUNK = 24;
    // the TMA box of a plane: x from ox-4 (a 16-byte boundary) to ox+35, y
    // from oy-2 to oy+9, the five conserved planes rho .. rho E
    static constexpr int BX = TX + 8, BY = PY, BV = 5;
    static constexpr int BOXF = BX * BY * BV;
    static constexpr int XFER = K * 5 * THREADS > BOXF ? K * 5 * THREADS : BOXF;   // floats of the fetch slot
};
static_assert((Gas3T::BOXF * 4) % 128 == 0, "the TMA box keeps 128-byte multiples");

// primitives (rho, u, v, w) and p of one cell or face value
struct __align__(128) Gas3Smem {
    // the fetch slot of the next plane, first (a tensor copy's destination
    // is 128-byte aligned): its TMA box [v][y][x], or per thread the conserved
    // values of its cells (asynchronous copies read back by the same thread)
    float xfer[Gas3T::XFER];
    unsigned long long mbar;                             // completion of the slot's tensor copy
    float4 pa[Gas3T::RING][Gas3T::PY][Gas3T::PX + 1];   // odd row length: column reads conflict-free
    float pp[Gas3T::RING][Gas3T::PY][Gas3T::PX + 1];
    float4 fvxa[Gas3T::TY][Gas3T::FXS];                  // right-face values, column -1 .. TX-1
    float fvxp[Gas3T::TY][Gas3T::FXS];
    float4 fvya[Gas3T::FYS][Gas3T::TX];                  // top-face values, row -1 .. TY-1
    float fvyp[Gas3T::FYS][Gas3T::TX];
    float4 hrxa[Gas3T::TY];                              // left-face values of column TX
    float hrxp[Gas3T::TY];
    float4 hrya[Gas3T::TX];                              // bottom-face values of row TY
    float hryp[Gas3T::TX];
    float4 fxa[Gas3T::TY][Gas3T::FXS];                   // x-face fluxes (rho, rho u, rho v, rho w)
    float fxe[Gas3T::TY][Gas3T::FXS];                    //  and rho E
    float4 fya[Gas3T::FYS][Gas3T::TX];
    float fye[Gas3T::FYS][Gas3T::TX];
    // per column: the carried top z-face value and bottom z-face flux
    float zcarry[10][Gas3T::CELLS];
    double red[32];
};

struct Gas3Args {
    const float *in;    // stage input
    const float *un;    // U^n
    float *out;         // stage output
    Ctl *ctl;
    int n0, n1, n2;
    long long pitch;
    float idx, idy, idz;
    int wall[3][2];     // reflective sides
    int zc;             // planes per CTA
    float Gam, invGam, pref0;
};

// HLLC flux of the gas with normal velocity un and tangential ut1, ut2
// (Sec. 3.1: Toro's HLLC, Davis wave speeds); F = (rho, normal momentum,
// tangential momenta 1 and 2, energy).
__device__ __forceinline__ void gas_hllc3(const Gas3Args &a, const float L[5], const float R[5], float F[5])
{
    // L, R: (rho, un, ut1, ut2, p)
    const float rL = L[0], unL = L[1], pL = L[4], rR = R[0], unR = R[1], pR = R[4];
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
    const int region = SL >= 0.f ? 0 : (Ss >= 0.f ? 1 : (SR > 0.f ? 2 : 3));
    const bool left = region <= 1, star = region == 1 || region == 2;
    // the upwind side's state, element by element (a pointer choice would
    // put both arrays in local memory)
    const float r = left ? L[0] : R[0], un = left ? L[1] : R[1], u1 = left ? L[2] : R[2];
    const float u2 = left ? L[3] : R[3], p = left ? L[4] : R[4];
    const float S = left ? SL : SR;
    const float E = (p - a.pref0) * a.invGam + 0.5f * r * un * un + 0.5f * r * u1 * u1 + 0.5f * r * u2 * u2;
    const float m = r * un;
    float Fr = m, Fn = m * un + p, F1 = m * u1, F2 = m * u2, FE = (E + p) * un;
    if (star) {
        const float iD = __fdividef(1.f, S - Ss);
        const float chi = (S - un) * iD;
        const float rs = r * chi;
        const float Es = chi * E + (Ss - un) * (rs * Ss + p * iD);
        Fr += S * (rs - r);
        Fn += S * (rs * Ss - m);
        F1 += S * (rs * u1 - r * u1);
        F2 += S * (rs * u2 - r * u2);
        FE += S * (Es - E);
    }
    F[0] = Fr;
    F[1] = Fn;
    F[2] = F1;
    F[3] = F2;
    F[4] = FE;
}

// A plane (with its x, y halo) in flight: its conserved values arrive in the
// fetch slot, by one tensor copy (TMA) or by every thread's asynchronous
// copies; the mirror flags of a thread's cells (3 bits each, cp.async path)
// or of the plane (TMA path) and the copy's mbarrier phase stay in registers.
struct Gas3Plane {
    unsigned flip;
    int gz;           // plane read
    unsigned phase;   // tensor copies issued so far (TMA path)
};

__device__ __forceinline__ void gas3_cp4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// One 4-D tensor copy (x, y, plane z, variable) of a box into shared memory.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int v,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int gas3_map(int i, int n, int wlo, int whi, bool *flip)
{
    if (i < 0) {
        if (wlo) {
            *flip = true;
            const int m = -1 - i;
            return m > n - 1 ? n - 1 : m;
        }
        return 0;
    }
    if (i > n - 1) {
        if (whi) {
            *flip = true;
            const int m = 2 * n - 1 - i;
            return m < 0 ? 0 : m;
        }
        return n - 1;
    }
    return i;
}

// loaded cell q of a plane -> (lx, ly) relative to the column's corner
__device__ __forceinline__ void gas3_cell(int q, int &lx, int &ly)
{
    using T = Gas3T;
    if (q < T::TY * T::PX) {
        ly = q / T::PX;
        lx = q - ly * T::PX - T::H;
    } else {
        const int r = q - T::TY * T::PX;
        const int row = r / T::TX;
        lx = r - row * T::TX;
        ly = row < 2 ? row - 2 : T::TY + (row - 2);
    }
}

// Start the fetch of plane z into the slot.  TMA: thread 0 issues one tensor
// copy of the box (the slot's previous contents have been read: the caller
// fetches after a barrier); otherwise every thread copies its own cells.
template <bool TMA>
__device__ __forceinline__ void gas3_fetch(const Gas3Args &a, const CUtensorMap *map, Gas3Smem &S, Gas3Plane &f,
                                           int ox, int oy, int z, bool interior)
{
    using T = Gas3T;
    bool fz = false;
    const int gz = gas3_map(z, a.n2, a.wall[2][0], a.wall[2][1], &fz);
    if constexpr (TMA) {
        f.flip = fz ? 4u : 0u;
        f.gz = gz;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&S.mbar, 4u * T::BOXF);
            tma_load_4d(S.xfer, map, ox - 4, oy - T::H, gz, 0, &S.mbar);
        }
        return;
    }
    f.flip = 0u;
#pragma unroll
    for (int k = 0; k < T::K; k++) {
        const int q = threadIdx.x + k * T::THREADS;
        if (q >= T::NCONV) continue;
        int lx, ly;
        gas3_cell(q, lx, ly);
        bool fx = false, fy = false;
        int gx = ox + lx, gy = oy + ly;
        if (!interior) {
            gx = gas3_map(gx, a.n0, a.wall[0][0], a.wall[0][1], &fx);
            gy = gas3_map(gy, a.n1, a.wall[1][0], a.wall[1][1], &fy);
        }
        f.flip |= ((fx ? 1u : 0u) | (fy ? 2u : 0u) | (fz ? 4u : 0u)) << (3 * k);
        const long long c = gx + (long long)a.n0 * (gy + (long long)a.n1 * gz);
#pragma unroll
        for (int v = 0; v < 5; v++) gas3_cp4(&S.xfer[(k * 5 + v) * T::THREADS + threadIdx.x], a.in + c + v * a.pitch);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void gas3_prim(const Gas3Args &a, const float q[5], unsigned flip, float w[5])
{
    const float ir = __fdividef(1.f, q[0]);
    const float u = q[1] * ir, v = q[2] * ir, ww = q[3] * ir;
    const float ke = 0.5f * q[0] * u * u + 0.5f * q[0] * v * v + 0.5f * q[0] * ww * ww;
    w[0] = q[0];
    w[1] = (flip & 1u) ? -u : u;
    w[2] = (flip & 2u) ? -v : v;
    w[3] = (flip & 4u) ? -ww : ww;
    w[4] = a.pref0 + a.Gam * (q[4] - ke);
}

// Convert the fetched plane into ring slot `slot`; false when a tensor copy
// never completed (bounded wait).
template <bool TMA>
__device__ __forceinline__ bool gas3_commit(const Gas3Args &a, Gas3Plane &f, Gas3Smem &S, int slot, int ox, int oy,
                                            bool interior)
{
    using T = Gas3T;
    if constexpr (TMA) {
        const bool ok = mbar_wait(&S.mbar, f.phase & 1u);
        f.phase++;
        if (!ok) return false;
    } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // this thread's copies have landed
    }
#pragma unroll
    for (int k = 0; k < T::K; k++) {
        const int q = threadIdx.x + k * T::THREADS;
        if (q >= T::NCONV) continue;
        int lx, ly;
        gas3_cell(q, lx, ly);
        float c5[5], w[5];
        unsigned flip;
        if constexpr (TMA) {
            // the cell's place in the box: the halo beyond a side is the
            // nearest cell or the mirror image (flip), clamped into the box
            // (cells far outside a small grid feed only faces outside it)
            bool fx = false, fy = false;
            int gx = ox + lx, gy = oy + ly;
            if (!interior) {
                gx = gas3_map(gx, a.n0, a.wall[0][0], a.wall[0][1], &fx);
                gy = gas3_map(gy, a.n1, a.wall[1][0], a.wall[1][1], &fy);
            }
            const int bx = min(max(gx - (ox - 4), 0), T::BX - 1), by = min(max(gy - (oy - T::H), 0), T::BY - 1);
#pragma unroll
            for (int v = 0; v < 5; v++) c5[v] = S.xfer[(v * T::BY + by) * T::BX + bx];
            flip = (fx ? 1u : 0u) | (fy ? 2u : 0u) | f.flip;
        } else {
#pragma unroll
            for (int v = 0; v < 5; v++) c5[v] = S.xfer[(k * 5 + v) * T::THREADS + threadIdx.x];
            flip = (f.flip >> (3 * k)) & 7u;
        }
        gas3_prim(a, c5, flip, w);
        S.pa[slot][ly + T::H][lx + T::H] = make_float4(w[0], w[1], w[2], w[3]);
        S.pp[slot][ly + T::H][lx + T::H] = w[4];
    }
    return true;
}

// primitives of the column's own cell in a ring slot
__device__ __forceinline__ void gas3_own(const Gas3Smem &S, int slot, int px, int py, float w[5])
{
    const float4 a4 = S.pa[slot][py][px];
    w[0] = a4.x;
    w[1] = a4.y;
    w[2] = a4.z;
    w[3] = a4.w;
    w[4] = S.pp[slot][py][px];
}

// primitives of the own column's cell at plane z, loaded and converted
// directly (the planes below the chunk, needed for its first z slopes only)
__device__ __forceinline__ void gas3_column(const Gas3Args &a, int gx, int gy, int z, float w[5])
{
    bool fz = false, fx = false, fy = false;
    const int gz = gas3_map(z, a.n2, a.wall[2][0], a.wall[2][1], &fz);
    const int cx = gas3_map(gx, a.n0, 0, 0, &fx), cy = gas3_map(gy, a.n1, 0, 0, &fy);
    const long long c = cx + (long long)a.n0 * (cy + (long long)a.n1 * gz);
    float q[5];
#pragma unroll
    for (int v = 0; v < 5; v++) q[v] = a.in[c + v * a.pitch];
    gas3_prim(a, q, fz ? 4u : 0u, w);
}

__device__ __forceinline__ void gas3_slope(const float m[5], const float c[5], const float p[5], float lo[5],
                                           float hi[5])
{
#pragma unroll
    for (int v = 0; v < 5; v++) {
        const float s = gas_vanleer(c[v] - m[v], p[v] - c[v]);
        lo[v] = c[v] - 0.5f * s;
        hi[v] = c[v] + 0.5f * s;
    }
}

// a face state in the order (rho, normal velocity, tangential 1, 2, p) for direction d
__device__ __forceinline__ void gas3_orient(const float w[5], int d, float o[5])
{
    o[0] = w[0];
    o[1] = w[1 + d];
    o[2] = w[1 + (d + 1) % 3];
    o[3] = w[1 + (d + 2) % 3];
    o[4] = w[4];
}

// flux in the order of orient back to (rho, rho u, rho v, rho w, rho E)
__device__ __forceinline__ void gas3_unorient(const float F[5], int d, float o[5])
{
    o[0] = F[0];
    o[1 + d] = F[1];
    o[1 + (d + 1) % 3] = F[2];
    o[1 + (d + 2) % 3] = F[3];
    o[4] = F[4];
}

// A tensor copy that did not complete in the bounded wait: report it, and
// give it one more bounded wait before the CTA's shared memory is released.
__device__ __forceinline__ void gas3_fail(const Gas3Args &a, Gas3Smem &S, const Gas3Plane &f)
{
    if (threadIdx.x == 0) {
        atomicOr(&a.ctl->err, (unsigned)ERR_TIMEOUT);
        (void)mbar_wait(&S.mbar, (f.phase - 1u) & 1u);
    }
}

// TMA: the plane boxes come by tensor copies through `map` (over the stage
// input's first five planes); else by per-thread asynchronous copies.
template <int STAGE, bool TMA>
__global__ void __launch_bounds__(Gas3T::THREADS, 3) k_gas3_stage(Gas3Args a, const __grid_constant__ CUtensorMap map)
{
    pdl_enter();
    using T = Gas3T;
    // the dynamic shared memory is the kernel's only shared memory and starts
    // the CTA's shared window; a tensor copy needs its slot 128-byte aligned
    extern __shared__ __align__(128) unsigned char gas3_smem_raw[];
    Gas3Smem &S = *reinterpret_cast<Gas3Smem *>(gas3_smem_raw);
    const int tid = threadIdx.x;
    if (TMA) {
        if ((smem_u32(S.xfer) & 127u) != 0) {
            // never issue a misaligned tensor copy: report and stop
            if (tid == 0) atomicOr(&a.ctl->err, (unsigned)ERR_TIMEOUT);
            return;
        }
        if (tid == 0) {
            mbar_init(&S.mbar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    const int ox = blockIdx.x * T::TX, oy = blockIdx.y * T::TY;
    const int z0 = blockIdx.z * a.zc, z1 = min(z0 + a.zc, a.n2);
    const bool interior = ox >= T::H && ox + T::TX + T::H <= a.n0 && oy >= T::H && oy + T::TY + T::H <= a.n1;
    const bool own = tid < T::CELLS;
    const int ci = tid & 31, cj = tid >> 5;
    const int gx = ox + ci, gy = oy + cj;
    const bool col = own && gx < a.n0 && gy < a.n1;
    const int px = ci + T::H, py = cj + T::H;
    const float dt = ctl_dt<float>(a.ctl);
    const float ca = STAGE == 2 ? 0.75f : (STAGE == 3 ? 1.f / 3.f : 0.f);
    const float cb = STAGE == 2 ? 0.25f : (STAGE == 3 ? 2.f / 3.f : 1.f);
    if (STAGE == 2 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) ctl_box_reset(a.ctl);

    // prologue: planes z0, z0+1 into the ring, plane z0+2 into registers
    // (committed by the first plane's step 1);
    // the column's planes z0-2, z0-1 for its first z slopes
    Gas3Plane fp;
    fp.phase = 0u;
    gas3_fetch<TMA>(a, &map, S, fp, ox, oy, z0, interior);
    if (__syncthreads_or(!gas3_commit<TMA>(a, fp, S, z0 % T::RING, ox, oy, interior))) {
        gas3_fail(a, S, fp);
        return;
    }
    gas3_fetch<TMA>(a, &map, S, fp, ox, oy, z0 + 1, interior);
    if (__syncthreads_or(!gas3_commit<TMA>(a, fp, S, (z0 + 1) % T::RING, ox, oy, interior))) {
        gas3_fail(a, S, fp);
        return;
    }
    gas3_fetch<TMA>(a, &map, S, fp, ox, oy, z0 + 2, interior);
    if (own) {
        float wm2[5], wm1[5], w0[5], w1[5], lo[5], hi[5], hiM[5], A[5], B[5], F[5];
        gas3_column(a, gx, gy, z0 - 2, wm2);
        gas3_column(a, gx, gy, z0 - 1, wm1);
        gas3_own(S, z0 % T::RING, px, py, w0);
        gas3_own(S, (z0 + 1) % T::RING, px, py, w1);
        gas3_slope(wm2, wm1, w0, lo, hiM);   // plane z0-1: its top-face value hiM
        gas3_slope(wm1, w0, w1, lo, hi);     // plane z0: bottom-face value lo, top-face value hi
        gas3_orient(hiM, 2, A);
        gas3_orient(lo, 2, B);
        gas_hllc3(a, A, B, F);
        float Fzlo[5];
        gas3_unorient(F, 2, Fzlo);           // the bottom z face of plane z0
#pragma unroll
        for (int v = 0; v < 5; v++) {
            S.zcarry[v][tid] = hi[v];
            S.zcarry[5 + v][tid] = Fzlo[v];
        }
    }

    float smax_cell = 0.f;
    int zlo = 0x7fffffff, zhi = -1;
    for (int z = z0; z < z1; z++) {
        const int sz = z % T::RING, s1 = (z + 1) % T::RING, s2 = (z + 2) % T::RING;
        // 1. plane z+2 into the ring (its slot held plane z-1, whose last
        // readers are behind the previous plane's barriers); then, with the
        // fetch slot read by every thread, plane z+3 fetched into it
        if (__syncthreads_or(!gas3_commit<TMA>(a, fp, S, s2, ox, oy, interior))) {
            gas3_fail(a, S, fp);
            return;
        }
        if (z + 3 <= z1 + 1) gas3_fetch<TMA>(a, &map, S, fp, ox, oy, z + 3, interior);
        if (col && z + 1 < z1) {
            // the cell's stage input and U^n at the next plane into L1 (read
            // at that plane's update; no register or shared slot holds them)
            const long long cn = gx + (long long)a.n0 * (gy + (long long)a.n1 * (z + 1));
#pragma unroll
            for (int v = 0; v < 6; v++) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(a.in + cn + v * a.pitch));
                if (STAGE > 1) asm volatile("prefetch.global.L1 [%0];" ::"l"(a.un + cn + v * a.pitch));
            }
        }

        // 2. slopes: x and y of plane z (face values to shared memory), z of plane z+1
        float qRx[5], qRy[5], qRz1[5], qLz1[5];
        if (own) {
            float wc[5], ww[5], we[5], ws[5], wn[5], hi[5];
            gas3_own(S, sz, px, py, wc);
            gas3_own(S, sz, px - 1, py, ww);
            gas3_own(S, sz, px + 1, py, we);
            gas3_own(S, sz, px, py - 1, ws);
            gas3_own(S, sz, px, py + 1, wn);
            gas3_slope(ww, wc, we, qRx, hi);
            S.fvxa[cj][ci + 1] = make_float4(hi[0], hi[1], hi[2], hi[3]);
            S.fvxp[cj][ci + 1] = hi[4];
            gas3_slope(ws, wc, wn, qRy, hi);
            S.fvya[cj + 1][ci] = make_float4(hi[0], hi[1], hi[2], hi[3]);
            S.fvyp[cj + 1][ci] = hi[4];
            float w1[5], w2[5];
            gas3_own(S, s1, px, py, w1);
            gas3_own(S, s2, px, py, w2);
            gas3_slope(wc, w1, w2, qRz1, qLz1);
        } else {
            // the extra warp: lanes 0-7 the right-face values of column -1,
            // lanes 8-15 the left-face values of column TX; every lane the
            // top-face value of row -1 and the bottom-face value of row TY
            const int l = tid - T::CELLS;
            const bool west = l < T::TY, east = !west && l < 2 * T::TY;
            const int jh = west ? l : (east ? l - T::TY : 0);
            const int cx = west ? T::H - 1 : T::TX + T::H;
            float m[5], c0[5], p[5], lo[5], hi[5];
            gas3_own(S, sz, cx - 1, jh + T::H, m);
            gas3_own(S, sz, cx, jh + T::H, c0);
            gas3_own(S, sz, cx + 1, jh + T::H, p);
            gas3_slope(m, c0, p, lo, hi);
            if (west) {
                S.fvxa[jh][0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
                S.fvxp[jh][0] = hi[4];
            } else if (east) {
                S.hrxa[jh] = make_float4(lo[0], lo[1], lo[2], lo[3]);
                S.hrxp[jh] = lo[4];
            }
            gas3_own(S, sz, l + T::H, T::H - 2, m);
            gas3_own(S, sz, l + T::H, T::H - 1, c0);
            gas3_own(S, sz, l + T::H, T::H, p);
            gas3_slope(m, c0, p, lo, hi);
            S.fvya[0][l] = make_float4(hi[0], hi[1], hi[2], hi[3]);
            S.fvyp[0][l] = hi[4];
            gas3_own(S, sz, l + T::H, T::TY + T::H - 1, m);
            gas3_own(S, sz, l + T::H, T::TY + T::H, c0);
            gas3_own(S, sz, l + T::H, T::TY + T::H + 1, p);
            gas3_slope(m, c0, p, lo, hi);
            S.hrya[l] = make_float4(lo[0], lo[1], lo[2], lo[3]);
            S.hryp[l] = lo[4];
        }
        __syncthreads();

        // 3. faces: left x, bottom y, top z of the cell
        float Fxl[5], Fyl[5], Fzhi[5];
        if (own) {
            float A[5], B[5], F[5], Lw[5];
            {
                const float4 l4 = S.fvxa[cj][ci];
                const float Lv[5] = {l4.x, l4.y, l4.z, l4.w, S.fvxp[cj][ci]};
                gas3_orient(Lv, 0, A);
                gas3_orient(qRx, 0, B);
                gas_hllc3(a, A, B, F);
                gas3_unorient(F, 0, Fxl);
            }
            {
                const float4 l4 = S.fvya[cj][ci];
                const float Lv[5] = {l4.x, l4.y, l4.z, l4.w, S.fvyp[cj][ci]};
                gas3_orient(Lv, 1, A);
                gas3_orient(qRy, 1, B);
                gas_hllc3(a, A, B, F);
                gas3_unorient(F, 1, Fyl);
            }
#pragma unroll
            for (int v = 0; v < 5; v++) Lw[v] = S.zcarry[v][tid];
            gas3_orient(Lw, 2, A);
            gas3_orient(qRz1, 2, B);
            gas_hllc3(a, A, B, F);
            gas3_unorient(F, 2, Fzhi);
            S.fxa[cj][ci] = make_float4(Fxl[0], Fxl[1], Fxl[2], Fxl[3]);
            S.fxe[cj][ci] = Fxl[4];
            S.fya[cj][ci] = make_float4(Fyl[0], Fyl[1], Fyl[2], Fyl[3]);
            S.fye[cj][ci] = Fyl[4];
        } else {
            const int l = tid - T::CELLS, jh = l < T::TY ? l : 0;
            float A[5], B[5], F[5], o[5];
            if (l < T::TY) {
                const float4 l4 = S.fvxa[jh][T::TX], r4 = S.hrxa[jh];
                const float Lv[5] = {l4.x, l4.y, l4.z, l4.w, S.fvxp[jh][T::TX]};
                const float Rv[5] = {r4.x, r4.y, r4.z, r4.w, S.hrxp[jh]};
                gas3_orient(Lv, 0, A);
                gas3_orient(Rv, 0, B);
                gas_hllc3(a, A, B, F);
                gas3_unorient(F, 0, o);
                S.fxa[jh][T::TX] = make_float4(o[0], o[1], o[2], o[3]);
                S.fxe[jh][T::TX] = o[4];
            }
            const float4 l4 = S.fvya[T::TY][l], r4 = S.hrya[l];
            const float Lv[5] = {l4.x, l4.y, l4.z, l4.w, S.fvyp[T::TY][l]};
            const float Rv[5] = {r4.x, r4.y, r4.z, r4.w, S.hryp[l]};
            gas3_orient(Lv, 1, A);
            gas3_orient(Rv, 1, B);
            gas_hllc3(a, A, B, F);
            gas3_unorient(F, 1, o);
            S.fya[T::TY][l] = make_float4(o[0], o[1], o[2], o[3]);
            S.fye[T::TY][l] = o[4];
        }
        __syncthreads();

        // 4. update of plane z: the cell's stage input and step-start values
        // (loaded here, not held through the faces: three CTAs fit an SM)
        const long long c = gx + (long long)a.n0 * (gy + (long long)a.n1 * z);
        if (col) {
            float cin[6], cun[6];
#pragma unroll
            for (int v = 0; v < 6; v++) {
                cin[v] = a.in[c + v * a.pitch];
                cun[v] = a.un[c + v * a.pitch];
            }
            const float4 e4 = S.fxa[cj][ci + 1], n4 = S.fya[cj + 1][ci];
            const float Fxr[5] = {e4.x, e4.y, e4.z, e4.w, S.fxe[cj][ci + 1]};
            const float Fyr[5] = {n4.x, n4.y, n4.z, n4.w, S.fye[cj + 1][ci]};
            const bool masked = cun[5] > 0.5f;
            float o[6];
#pragma unroll
            for (int v = 0; v < 5; v++) {
                Acc<float> D;
                D.set((Fxr[v] - Fxl[v]) * a.idx);
                D.add((Fyr[v] - Fyl[v]) * a.idy);
                D.add((Fzhi[v] - S.zcarry[5 + v][tid]) * a.idz);
                o[v] = masked ? cun[v] : rk_combine<float>(STAGE, cun[v], cin[v], D, dt, ca, cb);
            }
            {
                // r: no flux without a moving body
                Acc<float> D;
                D.set(0.f);
                D.add(0.f);
                D.add(0.f);
                o[5] = rk_combine<float>(STAGE, cun[5], cin[5], D, dt, ca, cb);
            }
#pragma unroll
            for (int v = 0; v < 6; v++) a.out[c + v * a.pitch] = o[v];
            if (!(o[0] > 0.f) || !(o[4] == o[4])) atomicOr(&a.ctl->err, (unsigned)ERR_STATE);
            if (STAGE == 3) {
                if (o[5] > 0.5f) {
                    zlo = min(zlo, z);
                    zhi = max(zhi, z);
                }
                float w[5];
                gas3_prim(a, o, 0u, w);
                const float c2 = __fdividef(a.Gam * w[4] + (w[4] - a.pref0), w[0]);
                if (!(c2 > 0.f)) atomicOr(&a.ctl->err, (unsigned)ERR_SOUND);
                const float cs = sqrtf(c2);
                smax_cell = fmaxf(smax_cell,
                                  (fabsf(w[1]) + cs) * a.idx + (fabsf(w[2]) + cs) * a.idy + (fabsf(w[3]) + cs) * a.idz);
            }
        }
        if (own) {
#pragma unroll
            for (int v = 0; v < 5; v++) {
                S.zcarry[v][tid] = qLz1[v];
                S.zcarry[5 + v][tid] = Fzhi[v];
            }
        }
    }
    if (STAGE == 3) {
        // the column's rigid cells into the box of the next seeding, the
        // chunk's CFL maximum into the launch's running maximum
        const bool rig = zhi >= 0;
        if (__any_sync(0xffffffffu, rig)) {
            const int big = 0x7fffffff;
            const int b[6] = {rig ? gx : big, rig ? gy : big, rig ? zlo : big, rig ? gx : -1, rig ? gy : -1,
                              rig ? zhi : -1};
            int m[6];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                m[k] = __reduce_min_sync(0xffffffffu, b[k]);
                m[3 + k] = __reduce_max_sync(0xffffffffu, b[3 + k]);
            }
            if ((tid & 31) == 0) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    atomicMin(&a.ctl->rnext[k], m[k]);
                    atomicMax(&a.ctl->rnext[3 + k], m[3 + k]);
                }
            }
        }
        float *sr = reinterpret_cast<float *>(S.red);
        const float mx = block_max<T::THREADS, float>(smax_cell, sr);
        if (tid == 0) {
            double md = (double)mx;
            if (!(md >= 0.0)) md = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
            atomicMax(&a.ctl->smax_acc, (unsigned long long)__double_as_longlong(md));
        }
    }
}

// Host side (dfv_gas_f32_k.cu).
cudaError_t gas3_prepare();
// The tensor map of a stage input's first five planes (rho .. rho E) with the
// plane box of the kernel: 4-D (x, y, z, variable) over n0 x n1 x n2 x 5
// floats at base, row stride n0, plane stride n0 n1, variable stride pitch.
// False when the grid does not allow it (rows or planes not a multiple of 16
// bytes, a misaligned base); the kernel then copies per thread.
bool gas3_encode_map(CUtensorMap *map, const void *base, int n0, int n1, int n2, long long pitch);
// map: the stage input's tensor map, or nullptr for the per-thread copies.
cudaError_t gas3_stage(int stage, const Gas3Args &a, const CUtensorMap *map, cudaStream_t st);

}  // namespace dfv

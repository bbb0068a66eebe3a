// dfv_gas.cuh -- the SSP-RK3 stage (Sec. 3.1) of 2-D single-gas grids in FP32
// (ideal or stiffened gas, static body, transmissive or reflective sides):
// the form of the cylinder and of the batched ellipse workloads.
//
// One persistent kernel per stage serves single grids and batches: a CTA
// loops over (instance, tile) items, and while it computes one tile the
// conserved planes of its next tile (32 x 16 cells, a halo of 2, five planes)
// arrive in shared memory by one TMA tensor copy (cp.async.bulk.tensor, a
// tensor map over the instance's planes in this GPU's memory, completion on an
// mbarrier).  Per tile:
//   1. conversion: each loaded cell to primitives (rho, u, v, p) once;
//   2. slopes: each cell's van Leer slopes in x and y once, its two
//      right/top face values to shared memory, its left/bottom ones kept;
//   3. faces: each thread the HLLC flux of its cell's left x-face and bottom
//      y-face (an extra warp the tile's closing faces);
//   4. update: flux divergence with a compensated (TwoSum) sum, the rigid
//      mask, the RK combination, and in stage 3 the CFL maximum and the box of
//      the new rigid cells.
// Without a moving body the upwind r flux vanishes and r needs no
// reconstruction, so a halo of 2 suffices (MUSCL).  The arithmetic per face
// and per cell is that of the general stage kernel (dfv_kernels.cuh) written
// for one gas: p = p_ref + Gamma (rho E - rho |u|^2/2), c^2 = (Gamma p + p -
// p_ref)/rho (Sec. 2.1.2).
#pragma once

#include <cuda.h>

#include "dfv_kernels.cuh"

namespace dfv {

// one grid served by the gas stage kernel
struct GasInst {
    int n0, n1;
    int tiles_x, ntiles;
    long long off;       // element offset of the instance's planes
    long long pitch;     // elements between planes
    float idx, idy;      // 1/dx, 1/dy
    float dx, dy;
    int wall_x0, wall_x1, wall_y0, wall_y1;   // reflective sides
    Ctl *ctl;
    int rows;            // rows per chunk (the warp-marching kernel, dfv_gasw.cuh)
    int pad;
};

struct GasArgs {
    const GasInst *inst;
    const CUtensorMap *tmap;   // 4 per instance: the planes of U^n, U1, U3 (tile and halo),
                               // and of U^n again (the tile's own cells)
    const int2 *items;         // (instance, tile); nullptr: instance 0, tile = item
    long long nitems;
    unsigned int *queue;       // dynamic schedule counter (nullptr: static round-robin)
    const float *un;           // U^n (instance planes at inst.off)
    float *out;                // stage output
    float Gam, invGam, pref0;  // the gas: Gamma, 1/Gamma, constant p_ref
};

struct GasT {
    // 16 rows (one warp each) plus a warp for the halo work; 15 rows (16
    // warps, four per scheduler) measured no faster on the 256-ellipse batch
    // (ragged last tiles, the halo spread over fewer cells)
    static constexpr int TX = 32, TY = 8, H = 2;
    static constexpr int BX = TX + 8;          // TMA box width: x from ox-4 (16-byte aligned)
    static constexpr int BY = TY + 2 * H;      // box height: y from oy-2
    static constexpr int NP = 5;               // planes of the single-gas 2-D layout
    static constexpr int BOX = BX * BY;        // cells of one plane of the box
    static constexpr int PX = TX + 2 * H, PY = TY + 2 * H;   // primitives of the tile and halo
    static constexpr int CELLS = TX * TY;
    static constexpr int THREADS = CELLS + 32;               // + one warp for halo slopes and closing faces
    static constexpr int NCONV = TY * PX + 2 * H * TX;       // loaded cells needed (corners not)
    static constexpr int FXS = TX + 1;         // x-face arrays: columns -1 .. TX-1 (values) / 0 .. TX (fluxes)
    static constexpr int FYS = TY + 1;
    static constexpr unsigned BOX_BYTES = 4u * NP * BOX;
    static constexpr unsigned OWN_BYTES = 4u * NP * CELLS;   // U^n of the tile's own cells (stages 2, 3)
    static constexpr int NMAP = 4;                           // tensor maps per instance
    // a tensor copy's shared-memory destination must be 128-byte aligned:
    // every TMA buffer is padded to a multiple of 128 bytes
    static constexpr int TILE_FLOATS = (NP * BOX + 31) / 32 * 32;
    static constexpr int OWN_FLOATS = (NP * CELLS + 31) / 32 * 32;
};
static_assert((GasT::TILE_FLOATS * 4) % 128 == 0 && (GasT::OWN_FLOATS * 4) % 128 == 0,
              "TMA buffers must keep 128-byte alignment");

struct __align__(128) GasSmem {
    float tile[2][GasT::TILE_FLOATS];              // TMA destination, double-buffered (planes of BOX cells)
    float own[2][GasT::OWN_FLOATS];                // U^n of the tile's cells (stages 2, 3; TMA; planes of CELLS)
    // one float4 per cell or face (one 128-bit access): (rho, u, v, p) for
    // primitives and face values, (rho, rho u, rho v, rho E) for fluxes
    float4 prim[GasT::PY][GasT::PX + 1];           // tile and halo; odd row length: a column read is conflict-free
    float4 fvx[GasT::TY][GasT::FXS];               // right-face values q_{i+1/2}^L, column i = -1 .. TX-1
    float4 fvy[GasT::FYS][GasT::TX];               // top-face values, row j = -1 .. TY-1
    float4 hrx[GasT::TY];                          // left-face values of column TX (closing x faces)
    float4 hry[GasT::TX];                          // bottom-face values of row TY (closing y faces)
    float4 fx[GasT::TY][GasT::FXS];                // fluxes of x faces i-1/2, i = 0 .. TX
    float4 fy[GasT::FYS][GasT::TX];                // fluxes of y faces j-1/2, j = 0 .. TY
    double red[32];
    unsigned long long mbar[2];
    long long item[2];
    GasInst inst[2];                               // the instance record of each buffered item
    int2 w[2];                                     // (instance, tile) of each buffered item
};

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

// One 3-D tensor copy (x, y, plane) of a box into shared memory.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar))
        : "memory");
}

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

// Loaded cell (lx, ly) of the tile at (ox, oy) -> box index; the halo beyond
// a side is the nearest cell (transmissive) or the mirror image (wall; *fx,
// *fy set).  Cells far outside the grid (halo of a ragged tile) map to some
// loaded cell: they feed only faces outside the grid.
__device__ __forceinline__ int gas_box_index(const GasInst &I, int ox, int oy, int lx, int ly, bool *fx, bool *fy)
{
    int gx = ox + lx, gy = oy + ly;
    *fx = *fy = false;
    if (gx < 0) {
        if (I.wall_x0) {
            gx = -1 - gx;
            *fx = true;
        } else {
            gx = 0;
        }
    } else if (gx > I.n0 - 1) {
        if (I.wall_x1) {
            gx = 2 * I.n0 - 1 - gx;
            *fx = true;
        } else {
            gx = I.n0 - 1;
        }
    }
    if (gy < 0) {
        if (I.wall_y0) {
            gy = -1 - gy;
            *fy = true;
        } else {
            gy = 0;
        }
    } else if (gy > I.n1 - 1) {
        if (I.wall_y1) {
            gy = 2 * I.n1 - 1 - gy;
            *fy = true;
        } else {
            gy = I.n1 - 1;
        }
    }
    int bx = gx - (ox - 4), by = gy - (oy - GasT::H);
    bx = bx < 0 ? 0 : (bx > GasT::BX - 1 ? GasT::BX - 1 : bx);
    by = by < 0 ? 0 : (by > GasT::BY - 1 ? GasT::BY - 1 : by);
    return by * GasT::BX + bx;
}

__device__ __forceinline__ long long gas_next(const GasArgs &a, long long cur, int k)
{
    if (!a.queue) return (long long)blockIdx.x + (long long)(k + 1) * gridDim.x;
    (void)cur;
    return (long long)atomicAdd(a.queue, 1u);
}

// Thread 0: record item `it` in buffer `slot` (its work item and instance
// record) and start the tensor copies of its planes into that buffer.
template <int STAGE>
__device__ __forceinline__ void gas_issue(const GasArgs &a, GasSmem &S, int slot, long long it)
{
    using T = GasT;
    S.item[slot] = it;
    if (it >= a.nitems) return;
    const int2 w = a.items ? a.items[it] : make_int2(0, (int)it);
    S.w[slot] = w;
    S.inst[slot] = a.inst[w.x];
    const GasInst &I = S.inst[slot];
    const int ox = (w.y % I.tiles_x) * T::TX, oy = (w.y / I.tiles_x) * T::TY;
    const CUtensorMap *m = a.tmap + T::NMAP * w.x;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&S.mbar[slot], T::BOX_BYTES + (STAGE > 1 ? T::OWN_BYTES : 0u));
    tma_load_3d(&S.tile[slot][0], m + (STAGE - 1), ox - 4, oy - T::H, 0, &S.mbar[slot]);
    if (STAGE > 1) tma_load_3d(&S.own[slot][0], m + 3, ox, oy, 0, &S.mbar[slot]);
}

// ------------------------------------------------------------ the stage

template <int STAGE>
__global__ void __launch_bounds__(GasT::THREADS, 4) k_gas_stage(GasArgs a)
{
    using T = GasT;
    // the dynamic shared memory is the kernel's only shared memory and starts
    // the CTA's shared window (used directly, so that every access compiles to
    // a shared-memory instruction); its alignment is checked below
    extern __shared__ __align__(128) unsigned char gas_smem_raw[];
    GasSmem &S = *reinterpret_cast<GasSmem *>(gas_smem_raw);
    const int tid = threadIdx.x;
    if ((smem_u32(&S.tile[0][0]) & 127u) != 0) {
        // never issue a misaligned tensor copy: report and stop
        if (tid == 0 && a.nitems > 0) atomicOr(&a.inst[0].ctl->err, (unsigned)ERR_TIMEOUT);
        return;
    }

    if (tid == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    pdl_enter();   // the previous kernel (its writes of the stage input) is complete
    if (tid == 0) gas_issue<STAGE>(a, S, 0, a.queue ? (long long)atomicAdd(a.queue, 1u) : (long long)blockIdx.x);
    __syncthreads();

    const float ca = STAGE == 2 ? 0.75f : (STAGE == 3 ? 1.f / 3.f : 0.f);
    const float cb = STAGE == 2 ? 0.25f : (STAGE == 3 ? 2.f / 3.f : 1.f);
    const int ci = tid & 31, cj = tid >> 5;   // the thread's cell (tid < CELLS)

    // No barrier ends an item: the next item's copies are started after its
    // first barrier, which every thread passes only when done with this one.
    for (int k = 0;; k++) {
        const int slot = k & 1;
        const long long it = S.item[slot];
        if (it >= a.nitems) break;
        const GasInst &I = S.inst[slot];
        const int tile = S.w[slot].y;
        const int ox = (tile % I.tiles_x) * T::TX, oy = (tile / I.tiles_x) * T::TY;
        const bool ok = mbar_wait(&S.mbar[slot], (unsigned)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            // a copy that never completed: report it and stop (no other copy is in flight)
            if (tid == 0) atomicOr(&I.ctl->err, (unsigned)ERR_TIMEOUT);
            break;
        }
        const float *tl = &S.tile[slot][0];
        const bool interior = ox >= 2 && ox + T::TX + 2 <= I.n0 && oy >= 2 && oy + T::TY + 2 <= I.n1;

        // 1. primitives of the tile and its halo (corners not needed)
        for (int q = tid; q < T::NCONV; q += T::THREADS) {
            int lx, ly;
            if (q < T::TY * T::PX) {
                ly = q / T::PX;
                lx = q - ly * T::PX - T::H;
            } else {
                const int r = q - T::TY * T::PX;
                const int row = r / T::TX;
                lx = r - row * T::TX;
                ly = row < 2 ? row - 2 : T::TY + (row - 2);
            }
            bool fx = false, fy = false;
            const int b = interior ? (ly + T::H) * T::BX + (lx + 4) : gas_box_index(I, ox, oy, lx, ly, &fx, &fy);
            float wv[4];
            gas_prim(a, tl[b], tl[T::BOX + b], tl[2 * T::BOX + b], tl[3 * T::BOX + b], wv);
            if (fx) wv[1] = -wv[1];
            if (fy) wv[2] = -wv[2];
            S.prim[ly + T::H][lx + T::H] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
        __syncthreads();
        // every thread is done with the previous item: its buffer takes the next one
        if (tid == 0) gas_issue<STAGE>(a, S, slot ^ 1, gas_next(a, it, k));

        // 2. slopes once per cell; right/top face values to shared memory
        float qRx[4], qRy[4];
        if (tid < T::CELLS) {
            const int py = cj + T::H, px = ci + T::H;
            const float4 c4 = S.prim[py][px], w4 = S.prim[py][px - 1], e4 = S.prim[py][px + 1];
            const float4 s4 = S.prim[py - 1][px], n4 = S.prim[py + 1][px];
            const float q[4] = {c4.x, c4.y, c4.z, c4.w}, qw[4] = {w4.x, w4.y, w4.z, w4.w};
            const float qe[4] = {e4.x, e4.y, e4.z, e4.w}, qs[4] = {s4.x, s4.y, s4.z, s4.w};
            const float qn[4] = {n4.x, n4.y, n4.z, n4.w};
            float lx4[4], ly4[4];
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const float sx = gas_vanleer(q[v] - qw[v], qe[v] - q[v]);
                const float sy = gas_vanleer(q[v] - qs[v], qn[v] - q[v]);
                lx4[v] = q[v] + 0.5f * sx;
                ly4[v] = q[v] + 0.5f * sy;
                qRx[v] = q[v] - 0.5f * sx;
                qRy[v] = q[v] - 0.5f * sy;
            }
            S.fvx[cj][ci + 1] = make_float4(lx4[0], lx4[1], lx4[2], lx4[3]);
            S.fvy[cj + 1][ci] = make_float4(ly4[0], ly4[1], ly4[2], ly4[3]);
        } else {
            // the extra warp: lanes 0 .. TY-1 the right-face values of column
            // -1, lanes TY .. 2TY-1 the left-face values of column TX (row
            // l mod TY); every lane the top-face value of row -1 and the
            // bottom-face value of row TY of column l
            const int l = tid - T::CELLS;
            const bool west = l < T::TY, east = !west && l < 2 * T::TY;
            const int jh = west ? l : (east ? l - T::TY : 0);
            const int col = west ? T::H - 1 : T::TX + T::H;
            const float4 a0 = S.prim[jh + T::H][col - 1], a1 = S.prim[jh + T::H][col], a2 = S.prim[jh + T::H][col + 1];
            const float4 b0 = S.prim[T::H - 2][l + T::H], b1 = S.prim[T::H - 1][l + T::H], b2 = S.prim[T::H][l + T::H];
            const float4 d0 = S.prim[T::TY + T::H - 1][l + T::H], d1 = S.prim[T::TY + T::H][l + T::H],
                         d2 = S.prim[T::TY + T::H + 1][l + T::H];
            const float A0[4] = {a0.x, a0.y, a0.z, a0.w}, A1[4] = {a1.x, a1.y, a1.z, a1.w}, A2[4] = {a2.x, a2.y, a2.z, a2.w};
            const float B0[4] = {b0.x, b0.y, b0.z, b0.w}, B1[4] = {b1.x, b1.y, b1.z, b1.w}, B2[4] = {b2.x, b2.y, b2.z, b2.w};
            const float D0[4] = {d0.x, d0.y, d0.z, d0.w}, D1[4] = {d1.x, d1.y, d1.z, d1.w}, D2[4] = {d2.x, d2.y, d2.z, d2.w};
            float ra[4], rb[4], rd[4];
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const float sa = gas_vanleer(A1[v] - A0[v], A2[v] - A1[v]);
                const float sb = gas_vanleer(B1[v] - B0[v], B2[v] - B1[v]);
                const float sd = gas_vanleer(D1[v] - D0[v], D2[v] - D1[v]);
                ra[v] = west ? A1[v] + 0.5f * sa : A1[v] - 0.5f * sa;
                rb[v] = B1[v] + 0.5f * sb;
                rd[v] = D1[v] - 0.5f * sd;
            }
            if (west) S.fvx[jh][0] = make_float4(ra[0], ra[1], ra[2], ra[3]);
            else if (east) S.hrx[jh] = make_float4(ra[0], ra[1], ra[2], ra[3]);
            S.fvy[0][l] = make_float4(rb[0], rb[1], rb[2], rb[3]);
            S.hry[l] = make_float4(rd[0], rd[1], rd[2], rd[3]);
        }
        __syncthreads();

        // 3. faces: the cell's left x face and bottom y face
        float Fxl[4], Fyl[4];
        if (tid < T::CELLS) {
            const float4 Lx = S.fvx[cj][ci], Ly = S.fvy[cj][ci];
            gas_hllc(a, Lx.x, Lx.y, Lx.z, Lx.w, qRx[0], qRx[1], qRx[2], qRx[3], Fxl);
            float G[4];
            gas_hllc(a, Ly.x, Ly.z, Ly.y, Ly.w, qRy[0], qRy[2], qRy[1], qRy[3], G);
            // y face: normal momentum is rho v, tangential rho u
            Fyl[0] = G[0];
            Fyl[1] = G[2];
            Fyl[2] = G[1];
            Fyl[3] = G[3];
            S.fx[cj][ci] = make_float4(Fxl[0], Fxl[1], Fxl[2], Fxl[3]);
            S.fy[cj][ci] = make_float4(Fyl[0], Fyl[1], Fyl[2], Fyl[3]);
        } else {
            const int l = tid - T::CELLS, jh = l < T::TY ? l : 0;
            float G[4];
            if (l < T::TY) {
                const float4 L = S.fvx[jh][T::TX], R = S.hrx[jh];
                gas_hllc(a, L.x, L.y, L.z, L.w, R.x, R.y, R.z, R.w, G);
                S.fx[jh][T::TX] = make_float4(G[0], G[1], G[2], G[3]);
            }
            const float4 L = S.fvy[T::TY][l], R = S.hry[l];
            gas_hllc(a, L.x, L.z, L.y, L.w, R.x, R.z, R.y, R.w, G);
            S.fy[T::TY][l] = make_float4(G[0], G[2], G[1], G[3]);
        }
        __syncthreads();

        // 4. divergence, rigid mask, RK combination
        Ctl *ctl = I.ctl;
        const float dt = ctl_dt<float>(ctl);
        const int gx = ox + ci, gy = oy + cj;
        const bool inside = tid < T::CELLS && gx < I.n0 && gy < I.n1;
        float smax_cell = 0.f;
        bool rigid_new = false;
        if (STAGE == 2 && tile == 0 && tid == 0) ctl_box_reset(ctl);
        if (inside) {
            const long long c = I.off + gx + (long long)I.n0 * gy;
            const long long P = I.pitch;
            const int bc = (cj + T::H) * T::BX + (ci + 4);
            // U^n at the cell: the stage input itself in stage 1, its own copy after
            const float *own = STAGE == 1 ? tl + bc : &S.own[slot][tid];
            const int ostr = STAGE == 1 ? T::BOX : T::CELLS;
            float o[5];
            const float unr = own[4 * ostr];
            const bool masked = unr > 0.5f;
            const float4 fe4 = S.fx[cj][ci + 1], fn4 = S.fy[cj + 1][ci];
            const float Fxr[4] = {fe4.x, fe4.y, fe4.z, fe4.w}, Fyr[4] = {fn4.x, fn4.y, fn4.z, fn4.w};
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const float unv = own[v * ostr];
                const float div = (Fxr[v] - Fxl[v]) * I.idx;
                const float dvy = (Fyr[v] - Fyl[v]) * I.idy;
                Acc<float> D;
                D.set(div);
                D.add(dvy);
                o[v] = masked ? unv : rk_combine<float>(STAGE, unv, tl[v * T::BOX + bc], D, dt, ca, cb);
            }
            {
                // r: no flux without a moving body
                Acc<float> D;
                D.set(0.f);
                D.add(0.f);
                o[4] = rk_combine<float>(STAGE, unr, tl[4 * T::BOX + bc], D, dt, ca, cb);
            }
#pragma unroll
            for (int v = 0; v < 5; v++) a.out[c + v * P] = o[v];
            if (!(o[0] > 0.f) || !(o[3] == o[3])) atomicOr(&ctl->err, (unsigned)ERR_STATE);
            if (STAGE == 3) {
                rigid_new = o[4] > 0.5f;
                float wv[4];
                gas_prim(a, o[0], o[1], o[2], o[3], wv);
                const float c2 = __fdividef(a.Gam * wv[3] + (wv[3] - a.pref0), wv[0]);
                if (!(c2 > 0.f)) atomicOr(&ctl->err, (unsigned)ERR_SOUND);
                const float cs = sqrtf(c2);
                smax_cell = (fabsf(wv[1]) + cs) * I.idx + (fabsf(wv[2]) + cs) * I.idy;
            }
        }
        if (STAGE == 3) {
            // box of the new state's rigid cells and the tile's CFL maximum
            if (__any_sync(0xffffffffu, rigid_new)) {
                const int big = 0x7fffffff;
                const int b6[4] = {rigid_new ? gx : big, rigid_new ? gy : big, rigid_new ? gx : -1,
                                   rigid_new ? gy : -1};
                const int mx0 = __reduce_min_sync(0xffffffffu, b6[0]), my0 = __reduce_min_sync(0xffffffffu, b6[1]);
                const int mx1 = __reduce_max_sync(0xffffffffu, b6[2]), my1 = __reduce_max_sync(0xffffffffu, b6[3]);
                if ((tid & 31) == 0) {
                    atomicMin(&ctl->rnext[0], mx0);
                    atomicMin(&ctl->rnext[1], my0);
                    atomicMin(&ctl->rnext[2], 0);
                    atomicMax(&ctl->rnext[3], mx1);
                    atomicMax(&ctl->rnext[4], my1);
                    atomicMax(&ctl->rnext[5], 0);
                }
            }
            float *sr = reinterpret_cast<float *>(S.red);
            const float m = block_max<T::THREADS, float>(smax_cell, sr);
            if (tid == 0) {
                double md = (double)m;
                if (!(md >= 0.0)) md = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
                atomicMax(&ctl->smax_acc, (unsigned long long)__double_as_longlong(md));
            }
        }
    }
}

}  // namespace dfv

namespace dfv {

// Host side (dfv_gas_f32_k.cu).
cudaError_t gas_prepare();                  // opt the kernels in to their shared memory
int gas_max_ctas_per_sm();                  // resident CTAs per SM of the stage kernels
cudaError_t gas_stage(int stage, const GasArgs &a, int grid, cudaStream_t st);
// The four tensor maps of one instance whose planes start `off` elements
// into each buffer: 3-D (x, y, plane) over n0 x n1 x 5 floats with row stride
// n0 and plane stride pitch; maps 0-2 over U^n, U1, U3 with the box of a tile
// and its halo (40 x 20 x 5), map 3 over U^n with the box of a tile (32 x 16 x 5).
bool gas_encode_maps(CUtensorMap maps[GasT::NMAP], const void *const bases[3], long long off, int n0, int n1,
                     long long pitch);

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

// dfv_gasw.cuh -- the SSP-RK3 stage (Sec. 3.1) of 2-D single-gas grids in
// FP32 (ideal or stiffened gas, static body, transmissive or reflective
// sides), marched by independent warps: the form of the cylinder and of the
// batched ellipse workloads.
//
// A work item is a strip of 28 columns and a chunk of rows of one instance.
// Its warp holds the strip in its 32 lanes, one column each, with the halo of
// 2 columns on either side in lanes 0-1 and 30-31, and marches up the chunk
// one row per iteration.  Everything a row needs from the rows around it
// stays in registers:
//   - the primitives (rho, u, v, p) of rows j, j+1, j+2 (row j+2 converted
//     from the conserved values loaded one iteration earlier; row j+3 is
//     loaded meanwhile);
//   - the top-face value of row j and the flux of face j-1/2, both from the
//     previous iteration.
// Per row j: the van Leer slope of row j+1 in y gives the y face j+1/2
// (HLLC); the slope of row j in x (the neighbours' primitives by warp
// shuffle) gives each lane the flux of its left x face, and its right one by
// a shuffle from the next lane; then the compensated (TwoSum) divergence, the
// rigid mask and the RK combination of the owned cells, and in stage 3 the
// CFL maximum and the box of the new rigid cells.  Each cell of a strip is
// converted and given its slopes once (plus four rows and two rows of y
// slopes per chunk), each face is solved once (plus one y face per chunk),
// and no shared memory or block barrier is involved: the warps of a CTA
// share nothing.  Without a moving body the upwind r flux vanishes and r is
// not reconstructed, so a halo of 2 suffices (MUSCL).  The arithmetic per
// face and per cell is that of the general stage kernel written for one gas
// (dfv_gas.cuh).
#pragma once

#include "dfv_gas.cuh"

namespace dfv {

struct GaswT {
    static constexpr int H = 2;              // halo columns on each side of a strip
    static constexpr int OWN = 32 - 2 * H;   // owned columns of a strip: lanes H .. 31 - H
    static constexpr int WARPS = 4;          // warps of a CTA (independent)
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int MIN_CTAS = 5;       // resident CTAs per SM the registers are sized for (stages 2, 3)
};

struct GaswArgs {
    const GasInst *inst;   // per instance: strips, items (strips x chunks), rows per chunk
    const int2 *items;     // (instance, strip + strips * chunk); nullptr: instance 0, item = index
    long long nitems;
    unsigned int *queue;   // dynamic schedule counter (nullptr: static round-robin over the warps)
    const float *in;       // stage input (U^n, U1, U3); an instance's planes start at inst.off
    const float *un;       // U^n
    float *out;            // stage output (U^n itself in stage 3)
    float Gam, invGam, pref0;
};

// Cell index of halo cell g of a line of n cells: the nearest cell beyond a
// transmissive side, the mirror image beyond a reflective one (flip set),
// clamped into the line (lines shorter than the halo).
__device__ __forceinline__ int gasw_map(int g, int n, int wall0, int wall1, bool &flip)
{
    flip = false;
    if (g < 0) {
        flip = wall0 != 0;
        g = wall0 ? -1 - g : 0;
    } else if (g > n - 1) {
        flip = wall1 != 0;
        g = wall1 ? 2 * n - 1 - g : n - 1;
    }
    return g < 0 ? 0 : (g > n - 1 ? n - 1 : g);
}

// rho, rho u, rho v, rho E of one cell (planes P apart)
__device__ __forceinline__ void gasw_load4(const float *p, long long P, float c[4])
{
    c[0] = __ldg(p);
    c[1] = __ldg(p + P);
    c[2] = __ldg(p + 2 * P);
    c[3] = __ldg(p + 3 * P);
}

// primitives of a loaded cell, the velocity mirrored across a reflective side
template <class A>
__device__ __forceinline__ float4 gasw_prim(const A &a, const float c[4], bool fx, bool fy)
{
    float w[4];
    gas_prim(a, c[0], c[1], c[2], c[3], w);
    return make_float4(w[0], fx ? -w[1] : w[1], fy ? -w[2] : w[2], w[3]);
}

// the (rho, u) and (v, p) halves of a state, for the packed FP32 units
__device__ __forceinline__ float2 gasw_lo(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 gasw_hi(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 gasw_cat(const float2 &l, const float2 &h) { return make_float4(l.x, l.y, h.x, h.y); }

// van Leer face values of cell c from its backward and forward differences
// db = c - m, df = p - c along one direction: lo at its face towards m, hi
// at its face towards p
__device__ __forceinline__ void gasw_faces_d(const float4 &c, const float4 &db, const float4 &df, float4 &lo,
                                             float4 &hi)
{
    const float2 s0 = gas_vanleer2(gasw_lo(db), gasw_lo(df)), s1 = gas_vanleer2(gasw_hi(db), gasw_hi(df));
    const float2 mh = make_float2(-0.5f, -0.5f), ph = make_float2(0.5f, 0.5f);
    lo = gasw_cat(__ffma2_rn(mh, s0, gasw_lo(c)), __ffma2_rn(mh, s1, gasw_hi(c)));
    hi = gasw_cat(__ffma2_rn(ph, s0, gasw_lo(c)), __ffma2_rn(ph, s1, gasw_hi(c)));
}

__device__ __forceinline__ float4 gasw_sub(const float4 &p, const float4 &q)
{
    return gasw_cat(gas_sub2(gasw_lo(p), gasw_lo(q)), gas_sub2(gasw_hi(p), gasw_hi(q)));
}

// the same from the neighbours m and p
__device__ __forceinline__ void gasw_faces(const float4 &m, const float4 &c, const float4 &p, float4 &lo, float4 &hi)
{
    gasw_faces_d(c, gasw_sub(c, m), gasw_sub(p, c), lo, hi);
}

// HLLC flux (rho, rho u, rho v, rho E) of an x face and of a y face
template <class A>
__device__ __forceinline__ float4 gasw_flux_x(const A &a, const float4 &L, const float4 &R)
{
    float F[4];
    gas_hllc(a, L.x, L.y, L.z, L.w, R.x, R.y, R.z, R.w, F);
    return make_float4(F[0], F[1], F[2], F[3]);
}
template <class A>
__device__ __forceinline__ float4 gasw_flux_y(const A &a, const float4 &L, const float4 &R)
{
    float G[4];
    gas_hllc(a, L.x, L.z, L.y, L.w, R.x, R.z, R.y, R.w, G);   // normal velocity v, tangential u
    return make_float4(G[0], G[2], G[1], G[3]);
}

__device__ __forceinline__ float4 gasw_shfl_up(const float4 &v)
{
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1),
                       __shfl_up_sync(0xffffffffu, v.z, 1), __shfl_up_sync(0xffffffffu, v.w, 1));
}
__device__ __forceinline__ float4 gasw_shfl_down(const float4 &v)
{
    return make_float4(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1),
                       __shfl_down_sync(0xffffffffu, v.z, 1), __shfl_down_sync(0xffffffffu, v.w, 1));
}

// two conserved variables of an owned cell: flux divergence (the x and y
// terms summed by TwoSum, the error kept as the low part), rigid mask, RK
// combination out = ca un + cb (in - dt (hi + lo)), the low part first
template <int STAGE>
__device__ __forceinline__ float2 gasw_update2(float2 unv, float2 inv, float2 fxl, float2 fxr, float2 fyl, float2 fyr,
                                              float2 idx, float2 idy, float2 mdt, float2 ca, float2 cb, bool masked)
{
    const float2 div = __fmul2_rn(gas_sub2(fxr, fxl), idx);
    const float2 dvy = __fmul2_rn(gas_sub2(fyr, fyl), idy);
    const float2 hi = __fadd2_rn(div, dvy);
    const float2 bp = gas_sub2(hi, div);
    const float2 err = __fadd2_rn(gas_sub2(div, gas_sub2(hi, bp)), gas_sub2(dvy, bp));
    const float2 lo = __fadd2_rn(make_float2(0.f, 0.f), err);
    const float2 y = __ffma2_rn(mdt, hi, __ffma2_rn(mdt, lo, inv));
    if (masked) return unv;
    return STAGE == 1 ? y : __ffma2_rn(cb, y, __fmul2_rn(ca, unv));
}

// the next work item of a warp from the dynamic queue (lane 0 takes it)
__device__ __forceinline__ long long gasw_take(unsigned int *queue, int lane)
{
    unsigned v = 0;
    if (lane == 0) v = atomicAdd(queue, 1u);
    return (long long)__shfl_sync(0xffffffffu, v, 0);
}

template <int STAGE>
__device__ __forceinline__ void gasw_item(const GaswArgs &a, const GasInst &I, int tile, int lane, float ca,
                                          float cb)
{
    using T = GaswT;
    const int n0 = I.n0, n1 = I.n1, rows = I.rows;
    const int strip = tile % I.strips, chunk = tile / I.strips;
    const int y0 = chunk * rows, yend = min(y0 + rows, n1);
    const int gx = strip * T::OWN - T::H + lane;
    const int wy0 = I.wall_y0, wy1 = I.wall_y1;
    bool fx;
    const int cx = gasw_map(gx, n0, I.wall_x0, I.wall_x1, fx);
    const bool owned = lane >= T::H && lane < 32 - T::H && gx < n0;   // then cx == gx
    const long long P = I.pitch, n0l = n0;
    const float *in = a.in + I.off + cx;
    const float *unp = a.un + I.off + cx;
    float *out = a.out + I.off + cx;
    Ctl *ctl = I.ctl;
    const float dt = ctl_dt<float>(ctl);
    const float idx = I.idx, idy = I.idy;
    if (STAGE == 2 && tile == 0 && lane == 0) ctl_box_reset(ctl);   // stage 3 folds the new box

    // stencil rows y0-2 .. y0+1, and row y0+2 in flight
    float4 Pa, Pb, P0, P1;
    {
        float c[4][4];
        bool f[4];
#pragma unroll
        for (int r = 0; r < 4; r++) gasw_load4(in + n0l * gasw_map(y0 - 2 + r, n1, wy0, wy1, f[r]), P, c[r]);
        Pa = gasw_prim(a, c[0], fx, f[0]);
        Pb = gasw_prim(a, c[1], fx, f[1]);
        P0 = gasw_prim(a, c[2], fx, f[2]);
        P1 = gasw_prim(a, c[3], fx, f[3]);
    }
    float ld[4];
    bool fld;
    gasw_load4(in + n0l * gasw_map(y0 + 2, n1, wy0, wy1, fld), P, ld);
    float unx[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // U^n of the next row to update (stages 2, 3)
    if (STAGE > 1 && owned)
#pragma unroll
        for (int v = 0; v < 5; v++) unx[v] = unp[n0l * y0 + v * P];

    float4 qT, FyB;
    {
        float4 lo, hi, qB;
        gasw_faces(Pa, Pb, P0, lo, qT);   // top-face value of row y0-1
        gasw_faces(Pb, P0, P1, qB, hi);   // bottom- and top-face values of row y0
        FyB = gasw_flux_y(a, qT, qB);     // face y0 - 1/2
        qT = hi;
    }

    float smax = 0.f;
    int bx0 = 0x7fffffff, by0 = 0x7fffffff, bx1 = -1, by1 = -1;
    for (int j = y0; j < yend; j++) {
        const float4 P2 = gasw_prim(a, ld, fx, fld);   // row j+2
        if (j + 3 <= yend + 1) gasw_load4(in + n0l * gasw_map(j + 3, n1, wy0, wy1, fld), P, ld);
        float cin[5], u5[5];
        if (owned) {
#pragma unroll
            for (int v = 0; v < 5; v++) cin[v] = __ldg(in + n0l * j + v * P);
        }
#pragma unroll
        for (int v = 0; v < 5; v++) u5[v] = STAGE == 1 ? cin[v] : unx[v];
        if (STAGE > 1 && owned && j + 1 < yend)
#pragma unroll
            for (int v = 0; v < 5; v++) unx[v] = unp[n0l * (j + 1) + v * P];

        // y face j + 1/2 from the slopes of row j+1
        float4 qB1, qT1;
        gasw_faces(P0, P1, P2, qB1, qT1);
        const float4 FyT = gasw_flux_y(a, qT, qB1);
        // x faces of row j
        // (forward difference to the next lane; the backward one is the previous lane's forward one)
        float4 qL, qR;
        const float4 dF = gasw_sub(gasw_shfl_down(P0), P0);
        gasw_faces_d(P0, gasw_shfl_up(dF), dF, qL, qR);
        const float4 FxL = gasw_flux_x(a, gasw_shfl_up(qR), qL);   // face i - 1/2
        const float4 FxR = gasw_shfl_down(FxL);                     // face i + 1/2

        if (owned) {
            const bool masked = u5[4] > 0.5f;
            const float2 idx2 = make_float2(idx, idx), idy2 = make_float2(idy, idy);
            const float2 mdt2 = make_float2(-dt, -dt), ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb);
            float o[5];
            const float2 o01 = gasw_update2<STAGE>(make_float2(u5[0], u5[1]), make_float2(cin[0], cin[1]),
                                                   gasw_lo(FxL), gasw_lo(FxR), gasw_lo(FyB), gasw_lo(FyT), idx2, idy2,
                                                   mdt2, ca2, cb2, masked);
            const float2 o23 = gasw_update2<STAGE>(make_float2(u5[2], u5[3]), make_float2(cin[2], cin[3]),
                                                   gasw_hi(FxL), gasw_hi(FxR), gasw_hi(FyB), gasw_hi(FyT), idx2, idy2,
                                                   mdt2, ca2, cb2, masked);
            o[0] = o01.x;
            o[1] = o01.y;
            o[2] = o23.x;
            o[3] = o23.y;
            {
                // r: no flux without a moving body
                Acc<float> D;
                D.set(0.f);
                D.add(0.f);
                o[4] = rk_combine<float>(STAGE, u5[4], cin[4], D, dt, ca, cb);
            }
            float *op = out + n0l * j;
#pragma unroll
            for (int v = 0; v < 5; v++) op[v * P] = o[v];
            if (!(o[0] > 0.f) || !(o[3] == o[3])) atomicOr(&ctl->err, (unsigned)ERR_STATE);
            if (STAGE == 3) {
                if (o[4] > 0.5f) {
                    bx0 = min(bx0, gx);
                    by0 = min(by0, j);
                    bx1 = max(bx1, gx);
                    by1 = max(by1, j);
                }
                float wv[4];
                gas_prim(a, o[0], o[1], o[2], o[3], wv);
                const float c2 = __fmul_rn(fmaf(a.Gam, wv[3], wv[3] - a.pref0), gas_rcp(wv[0]));
                if (!(c2 > 0.f)) atomicOr(&ctl->err, (unsigned)ERR_SOUND);
                const float cs = sqrtf(c2);
                smax = fmaxf(smax, fmaf(fabsf(wv[1]) + cs, idx, __fmul_rn(fabsf(wv[2]) + cs, idy)));
            }
        }
        P0 = P1;
        P1 = P2;
        qT = qT1;
        FyB = FyT;
    }
    if (STAGE == 3) {
        // the item's CFL maximum and box of new rigid cells
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        if (__any_sync(0xffffffffu, bx1 >= 0)) {
            bx0 = __reduce_min_sync(0xffffffffu, bx0);
            by0 = __reduce_min_sync(0xffffffffu, by0);
            bx1 = __reduce_max_sync(0xffffffffu, bx1);
            by1 = __reduce_max_sync(0xffffffffu, by1);
            if (lane == 0) {
                atomicMin(&ctl->rnext[0], bx0);
                atomicMin(&ctl->rnext[1], by0);
                atomicMin(&ctl->rnext[2], 0);
                atomicMax(&ctl->rnext[3], bx1);
                atomicMax(&ctl->rnext[4], by1);
                atomicMax(&ctl->rnext[5], 0);
            }
        }
        if (lane == 0) {
            double md = (double)smax;
            if (!(md >= 0.0)) md = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
            atomicMax(&ctl->smax_acc, (unsigned long long)__double_as_longlong(md));
        }
    }
}

template <int STAGE>
// stage 1 (no U^n stream of its own) fits in 80 registers: six CTAs per SM
__global__ void __launch_bounds__(GaswT::THREADS, STAGE == 1 ? 6 : GaswT::MIN_CTAS) k_gasw_stage(GaswArgs a)
{
    using T = GaswT;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * T::WARPS;
    long long it = (long long)blockIdx.x * T::WARPS + (threadIdx.x >> 5);
    const float ca = STAGE == 2 ? 0.75f : (STAGE == 3 ? 1.f / 3.f : 0.f);
    const float cb = STAGE == 2 ? 0.25f : (STAGE == 3 ? 2.f / 3.f : 1.f);
    pdl_enter();   // the previous kernel (its writes of the stage input) is complete
    if (a.queue) it = gasw_take(a.queue, lane);
    while (it < a.nitems) {
        // the next item is taken before this one runs (the queue's latency overlaps it)
        const long long next = a.queue ? gasw_take(a.queue, lane) : it + nw;
        const int2 w = a.items ? a.items[it] : make_int2(0, (int)it);
        gasw_item<STAGE>(a, a.inst[w.x], w.y, lane, ca, cb);
        it = next;
    }
}

// Host side (dfv_gas_f32_k.cu).
int gasw_max_ctas_per_sm();   // resident CTAs per SM of the stage kernels
cudaError_t gasw_stage(int stage, const GaswArgs &a, int grid, cudaStream_t st);
// Rows per chunk for grids of `cells` cells in all: long chunks (few repeated
// halo rows) while there are enough work items to keep every warp busy.
int gasw_rows(long long cells);
// Strips (28 columns) and items of one instance.
inline int gasw_strips(int n0) { return (n0 + GaswT::OWN - 1) / GaswT::OWN; }

}  // namespace dfv

// dfv_batch.cuh -- many independent 2-D instances (own grid size, body and
// time step) advanced together: every kernel is a persistent launch over a
// work list of (instance, tile) items, so one launch per phase serves the whole
// batch.  The per-tile work is the single-grid stage_tile / seeding code.
#pragma once

#include <algorithm>

#include "dfv_kernels.cuh"

namespace dfv {

struct BatchInst {
    GridP g;            // the instance's grid and materials (pitch: its own)
    long long off;      // element offset of its planes in the state arrays
    long long part0;    // its first slot in the partials array (4 doubles each)
    int tiles_x, tiles_y, ntiles, pad;
    Ctl *ctl;           // its control block (dt, t, smax, ticket, error word)
};

struct BatchArgs {
    const void *in;          // stage input, read with halo
    const void *un;          // U^n
    void *out;               // stage output
    const BatchInst *inst;
    const int2 *items;       // (instance, tile) in the order of the schedule
    long long nitems;
    double *partials;
    int final_mode;          // finalize mode: by each instance's last tile (CFL phase) or
                             // by the finalize phase after stage 3
    unsigned int *queue;     // dynamic schedule: next item counter (nullptr: static round-robin)
};

// Next work item of this CTA: static round-robin or a shared counter.
__device__ __forceinline__ long long next_item(const BatchArgs &b, long long cur, long long *s_item)
{
    if (!b.queue) return cur < 0 ? (long long)blockIdx.x : cur + gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) *s_item = (long long)atomicAdd(b.queue, 1u);
    __syncthreads();
    return *s_item;
}

// Copy the instance record into shared memory (GridP is read all through the
// tile code; shared memory keeps those reads off the global path).
__device__ __forceinline__ void load_inst(const BatchInst *src, BatchInst *dst)
{
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(dst);
    constexpr int NW = (int)(sizeof(BatchInst) / sizeof(int));
    for (int k = threadIdx.x; k < NW; k += blockDim.x) d[k] = s[k];
}

// Register bound: five CTAs per SM for the FP32 single-material form (40
// registers, a few dozen bytes of spills; 1 % faster than four on the
// 256-ellipse batch), two otherwise.
template <class R, int NMAT, int STAGE>
__global__ void __launch_bounds__(Tile<2, (int)sizeof(R)>::THREADS, (sizeof(R) == 4 && NMAT == 1) ? 5 : 2)
    k_batch_stage(BatchArgs b)
{
    pdl_enter();
    __shared__ BatchInst s_inst;
    __shared__ long long s_item;
    __shared__ int s_cur;
    if (threadIdx.x == 0) s_cur = -1;
    for (long long it = next_item(b, -1, &s_item); it < b.nitems; it = next_item(b, it, &s_item)) {
        const int2 w = b.items[it];
        __syncthreads();
        if (s_cur != w.x) {
            load_inst(&b.inst[w.x], &s_inst);
            __syncthreads();
            if (threadIdx.x == 0) s_cur = w.x;
        }
        __syncthreads();
        const BatchInst &I = s_inst;
        StageArgs a;
        a.in = reinterpret_cast<const R *>(b.in) + I.off;
        a.un = reinterpret_cast<const R *>(b.un) + I.off;
        a.out = reinterpret_cast<R *>(b.out) + I.off;
        a.ctl = I.ctl;
        a.partials = b.partials + 4 * I.part0;
        a.want_force = 0;
        a.early = 0;
        a.next = 0;
        stage_tile<R, 2, NMAT, false, STAGE>(I.g, a, w.y % I.tiles_x, w.y / I.tiles_x, 0, w.y, I.ntiles);
    }
}

// Rigid seeding of every instance: SEED_CTAS CTAs of 256 threads per
// instance stride over the cells of its rigid box (the whole grid until its
// first stage 3); the instance record is read through the cache.
// MODE 0: in place; 1: seeded states into the scratch planes b.out; 2: the
// scratch into U (the fixed probe reads the step-start state only).
constexpr int SEED_CTAS = 32;

template <class R, int NMAT, int MODE, int OPT>
__global__ void __launch_bounds__(256) k_batch_seed(BatchArgs b)
{
    pdl_enter();
    const BatchInst &I = b.inst[blockIdx.x / SEED_CTAS];
    R *U = reinterpret_cast<R *>(const_cast<void *>(b.in)) + I.off;
    R *S = reinterpret_cast<R *>(b.out) + I.off;
    seed_box_cells<R, 2, NMAT, false, OPT, MODE>(U, S, I.ctl, I.g,
                                                 (blockIdx.x % SEED_CTAS) * (long long)blockDim.x,
                                                 (long long)SEED_CTAS * blockDim.x, false);
}

// CFL wave speed of every instance's stored state; the last tile of each
// instance reduces its partials and sets its dt (b.final_mode).
template <class R, int NMAT>
__global__ void __launch_bounds__(Tile<2, (int)sizeof(R)>::THREADS) k_batch_cfl(BatchArgs b)
{
    using TL = Tile<2, (int)sizeof(R)>;
    using L = Lay<2, NMAT, false>;
    __shared__ BatchInst s_inst;
    __shared__ long long s_item;
    __shared__ int s_cur;
    __shared__ double sred[4 * 32];
    __shared__ unsigned int s_last;
    if (threadIdx.x == 0) s_cur = -1;
    for (long long it = next_item(b, -1, &s_item); it < b.nitems; it = next_item(b, it, &s_item)) {
        const int2 w = b.items[it];
        __syncthreads();
        if (s_cur != w.x) {
            load_inst(&b.inst[w.x], &s_inst);
            __syncthreads();
            if (threadIdx.x == 0) s_cur = w.x;
        }
        __syncthreads();
        const BatchInst &I = s_inst;
        double red[4] = {0.0, 0.0, 0.0, 0.0};
        if (threadIdx.x < TL::TX * TL::TY) {
            const int gx = (w.y % I.tiles_x) * TL::TX + threadIdx.x % TL::TX;
            const int gy = (w.y / I.tiles_x) * TL::TY + threadIdx.x / TL::TX;
            if (gx < I.g.n[0] && gy < I.g.n[1]) {
                const R *U = reinterpret_cast<const R *>(b.in) + I.off;
                const long long c = gx + (long long)I.g.n[0] * gy;
                R q[L::NVAR], wv[L::NVAR];
#pragma unroll
                for (int v = 0; v < L::NVAR; v++) q[v] = U[v * I.g.pitch + c];
                cons_to_prim<R, 2, NMAT, false>(I.g, q, wv);
                State<R, 2, NMAT, false> s;
                state_from_prim<R, 2, NMAT, false>(I.g, wv, s);
                const R cs = m_sqrt(s.c2);
                R sum = R(0);
#pragma unroll
                for (int d = 0; d < 2; d++) sum += (m_abs(s.u[d]) + cs) / gridc<R>(I.g).dx[d];
                double sd = (double)sum;
                if (!(sd == sd)) sd = __longlong_as_double(0x7ff0000000000000LL);
                red[0] = sd;
            }
        }
        block_reduce4<TL::THREADS>(red, sred);
        if (threadIdx.x == 0) {
            b.partials[4 * (I.part0 + w.y)] = red[0];
            __threadfence();
            const unsigned int t = atomicAdd(&I.ctl->ticket, 1u);
            s_last = (t == (unsigned int)(I.ntiles - 1)) ? 1u : 0u;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finalize_block<TL::THREADS>(I.ctl, b.partials + 4 * I.part0, I.ntiles, I.ntiles, b.final_mode, 2,
                                        I.g.dx[0], I.g.dx[1], I.g.dx[2], sred);
            if (threadIdx.x == 0) I.ctl->ticket = 0u;
        }
    }
}

// Finalize of every instance after stage 3, one block per instance: its CFL
// maximum (folded by its stage-3 tiles), time, step count and next dt.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch_finalize(BatchArgs b)
{
    pdl_enter();
    __shared__ double sred[4 * 32];
    const BatchInst &I = b.inst[blockIdx.x];
    finalize_block<THREADS>(I.ctl, b.partials + 4 * I.part0, 0, 0, b.final_mode, 2, I.g.dx[0], I.g.dx[1],
                            I.g.dx[2], sred);
    // the stages of this step are complete: reset the dynamic-schedule counters
    if (blockIdx.x == 0 && threadIdx.x == 0 && b.queue)
        for (int k = 1; k <= 3; k++) b.queue[k] = 0u;
}

static __global__ void k_batch_init_ctl(Ctl *ctl, int count, const double *v_body /* 3 per instance */)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        Ctl *c = ctl + i;
        memset(c, 0, sizeof(Ctl));
        ctl_box_reset(c);
        for (int d = 0; d < 3; d++) c->v[d] = v_body[3 * i + d];
        ctl_sync_v(c);
    }
}

static __global__ void k_batch_set_run(Ctl *ctl, int count, double cfl, double t_end)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        ctl[i].cfl = cfl;
        ctl[i].t_end = t_end;
    }
}

// Launch table of the batch kernels of one precision.
template <class R, int NMAT>
struct BK {
    static constexpr int threads = Tile<2, (int)sizeof(R)>::THREADS;
    static constexpr size_t smem = StageSmem<R, 2, NMAT, false>::bytes;
    static cudaError_t prepare()
    {
        cudaError_t e = cudaFuncSetAttribute(k_batch_stage<R, NMAT, 1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_stage<R, NMAT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_stage<R, NMAT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        return e;
    }
    static int max_ctas_per_sm()
    {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_stage<R, NMAT, 2>, threads, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_stage<R, NMAT, 3>, threads, smem);
        return std::max(1, std::min(a, b));
    }
    template <int MODE>
    static void seed(int opt, int grid, const BatchArgs &a, cudaStream_t st)
    {
        switch (opt) {
        case 0: launch_pdl(k_batch_seed<R, NMAT, MODE, 0>, dim3(grid * SEED_CTAS), dim3(256), 0, st, a); break;
        case 1: launch_pdl(k_batch_seed<R, NMAT, MODE, 1>, dim3(grid * SEED_CTAS), dim3(256), 0, st, a); break;
        case 2: launch_pdl(k_batch_seed<R, NMAT, MODE, 2>, dim3(grid * SEED_CTAS), dim3(256), 0, st, a); break;
        default: launch_pdl(k_batch_seed<R, NMAT, MODE, 3>, dim3(grid * SEED_CTAS), dim3(256), 0, st, a); break;
        }
    }
    // phase: 0 seed in place, 1..3 stages, 4 CFL, 5 / 6 seed to scratch / apply,
    // 7 finalize after stage 3;
    // opt: the seeding option set (seed_opt)
    static cudaError_t launch(int phase, int grid, const BatchArgs &a, int opt, cudaStream_t st)
    {
        switch (phase) {
        case 0: seed<0>(opt, grid, a, st); break;
        case 5: seed<1>(opt, grid, a, st); break;
        case 6: launch_pdl(k_batch_seed<R, NMAT, 2, 0>, dim3(grid * SEED_CTAS), dim3(256), 0, st, a); break;
        case 7: launch_pdl(k_batch_finalize<32>, dim3(grid), dim3(32), 0, st, a); break;
        case 1: launch_pdl(k_batch_stage<R, NMAT, 1>, dim3(grid), dim3(threads), smem, st, a); break;
        case 2: launch_pdl(k_batch_stage<R, NMAT, 2>, dim3(grid), dim3(threads), smem, st, a); break;
        case 3: launch_pdl(k_batch_stage<R, NMAT, 3>, dim3(grid), dim3(threads), smem, st, a); break;
        default: k_batch_cfl<R, NMAT><<<grid, threads, 0, st>>>(a); break;
        }
        return cudaGetLastError();
    }
};

struct Kern {
    cudaError_t (*prepare)();
    int (*max_ctas_per_sm)();
    cudaError_t (*launch)(int, int, const BatchArgs &, int, cudaStream_t);
};

template <class R>
Kern batch_kernels(int nmat)
{
    return nmat == 1   ? Kern{BK<R, 1>::prepare, BK<R, 1>::max_ctas_per_sm, BK<R, 1>::launch}
           : nmat == 2 ? Kern{BK<R, 2>::prepare, BK<R, 2>::max_ctas_per_sm, BK<R, 2>::launch}
                       : Kern{BK<R, 3>::prepare, BK<R, 3>::max_ctas_per_sm, BK<R, 3>::launch};
}

// One translation unit per precision (the FP32 one is built with the fast
// single-precision divide, like the single-grid FP32 kernels).
Kern batch_kernels_f32(int nmat);
Kern batch_kernels_f64(int nmat);


}  // namespace dfv

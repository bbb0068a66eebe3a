// dfv_inst.cuh -- builds the launcher table of one precision; included by
// dfv_inst_f64.cu and dfv_inst_f32.cu with R set to the storage type.
#pragma once

#include "dfv_kernels.cuh"
#include "dfv_kernels_z.cuh"
#include "dfv_ops.h"

namespace dfv {

template <class R, int DIM, int NMAT, int SOLID>
struct Impl {
    using L = Lay<DIM, NMAT, SOLID>;
    using TL = Tile<DIM, (int)sizeof(R)>;

    static dim3 stage_grid(const GridP &g)
    {
        return dim3((g.n[0] + TL::TX - 1) / TL::TX, (g.n[1] + TL::TY - 1) / TL::TY, (g.n[2] + TL::TZ - 1) / TL::TZ);
    }

    static constexpr size_t smem = StageSmem<R, DIM, NMAT, SOLID>::bytes;

    // 3-D FP32 single-material fluids march along z (k_stage_z); stage 1
    // with the pressure force keeps the tiled kernel, whose tiles own the
    // force partials
    static constexpr bool ZM = DIM == 3 && SOLID == 0 && NMAT == 1 && sizeof(R) == 4;
    static constexpr size_t zsmem = ZSmem<R, NMAT>::bytes;
    // planes per CTA: 32 on the 256^3 sphere beats 16, 24, 64 and 256 (the
    // six-plane prologue of a chunk against the CTA count for the 152 SMs)
    static constexpr int ZCHUNK = 32;

    static dim3 zgrid(const GridP &g)
    {
        return dim3((g.n[0] + ZGeo::TX - 1) / ZGeo::TX, (g.n[1] + ZGeo::TY - 1) / ZGeo::TY,
                    (g.n[2] + ZCHUNK - 1) / ZCHUNK);
    }

    // Opt the stage kernels in to their dynamic shared memory on the current
    // device (called at grid creation, outside any stream capture).
    static cudaError_t prepare()
    {
        cudaError_t e = cudaFuncSetAttribute(k_stage<R, DIM, NMAT, SOLID, 1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stage<R, DIM, NMAT, SOLID, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stage<R, DIM, NMAT, SOLID, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        // the first-wave size is looked up here, outside any stream capture
        if (e == cudaSuccess) (void)first_wave();
        if constexpr (ZM) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_stage_z<R, NMAT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zsmem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_stage_z<R, NMAT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zsmem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_stage_z<R, NMAT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zsmem);
        }
        return e;
    }

    template <int S>
    static cudaError_t stage_s(const GridP &g, const StageArgs &a, cudaStream_t st)
    {
        if constexpr (ZM) {
            if (!(S == 1 && a.want_force))
                return launch_pdl(k_stage_z<R, NMAT, S>, zgrid(g), dim3(ZGeo::THREADS), zsmem, st, a, g, ZCHUNK);
        }
        return launch_pdl(k_stage<R, DIM, NMAT, SOLID, S>, stage_grid(g), dim3(TL::THREADS), smem, st, a, g);
    }

    // CTAs of the stage-1 kernel resident at once on the device (the first
    // wave), looked up once
    static int first_wave()
    {
        static int n = -1;
        if (n < 0) {
            int dev = 0, sms = 0, per = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage<R, DIM, NMAT, SOLID, 1>, TL::THREADS,
                                                              smem) != cudaSuccess) {
                (void)cudaGetLastError();
                return 0;
            }
            n = sms * per;
        }
        return n;
    }

    // next: the seeding before stage 1 reads its box from ctl->rnext
    static cudaError_t stage(int s, const GridP &g, const void *in, const void *un, void *out, Ctl *ctl,
                             double *partials, int want_force, int next, cudaStream_t st)
    {
        StageArgs a;
        a.in = in;
        a.un = un;
        a.out = out;
        a.ctl = ctl;
        a.partials = partials;
        a.want_force = want_force;
        a.early = s == 1 ? first_wave() : 0;
        a.next = next;
        if (s == 1) return stage_s<1>(g, a, st);
        if (s == 2) return stage_s<2>(g, a, st);
        return stage_s<3>(g, a, st);
    }

    template <int OPT>
    static cudaError_t seed_opt_k(const GridP &g, void *U, void *scratch, Ctl *ctl, int fin_mode, cudaStream_t st)
    {
        dim3 block, grid;
        seed_grid(g, block, grid);
        if (g.probe_mode == 1) {
            cudaError_t e = launch_pdl(k_seed<R, DIM, NMAT, SOLID, OPT, 1>, grid, block, 0, st, U, scratch, ctl, g, 0);
            if (e != cudaSuccess) return e;
            return launch_pdl(k_seed<R, DIM, NMAT, SOLID, 0, 2>, grid, block, 0, st, U, scratch, ctl, g, 0);
        }
        if (fin_mode) grid.x += 1;   // the block that runs the deferred finalize
        return launch_pdl(k_seed<R, DIM, NMAT, SOLID, OPT, 0>, grid, block, 0, st, U, scratch, ctl, g, fin_mode);
    }

    // seeding; scratch: planes of the grid's layout free until stage 1;
    // fin_mode: the deferred finalize of the previous step (stepped probe
    // only), 0 for none
    static cudaError_t seed(const GridP &g, void *U, void *scratch, Ctl *ctl, int fin_mode, cudaStream_t st)
    {
        switch (seed_opt(g)) {
        case 0: return seed_opt_k<0>(g, U, scratch, ctl, fin_mode, st);
        case 1: return seed_opt_k<1>(g, U, scratch, ctl, fin_mode, st);
        case 2: return seed_opt_k<2>(g, U, scratch, ctl, fin_mode, st);
        default: return seed_opt_k<3>(g, U, scratch, ctl, fin_mode, st);
        }
    }

    static cudaError_t cfl(const GridP &g, const void *U, double *partials, int nblocks, cudaStream_t st)
    {
        k_cfl<R, DIM, NMAT, SOLID><<<nblocks, 256, 0, st>>>(U, partials, g);
        return cudaGetLastError();
    }

    static cudaError_t p2c(const GridP &g, const double *prim, long long pp, void *U, cudaStream_t st)
    {
        k_prim_to_cons<R, DIM, NMAT, SOLID><<<gs_blocks(g.ncell), 256, 0, st>>>(prim, pp, U, g);
        return cudaGetLastError();
    }

    static cudaError_t c2p(const GridP &g, const void *U, double *prim, long long pp, cudaStream_t st)
    {
        k_cons_to_prim<R, DIM, NMAT, SOLID><<<gs_blocks(g.ncell), 256, 0, st>>>(U, prim, pp, g);
        return cudaGetLastError();
    }

    static cudaError_t c2f(const GridP &g, const void *U, double *o, long long pp, int nvar, cudaStream_t st)
    {
        k_cons_to_f64<R><<<gs_blocks(g.ncell), 256, 0, st>>>(U, o, pp, nvar, g);
        return cudaGetLastError();
    }

    static const Ops *ops()
    {
        static const Ops o = {L::NVAR, TL::THREADS, (int)sizeof(R), &prepare, &stage_grid, &seed, &stage, &cfl,
                              &p2c, &c2p, &c2f};
        return &o;
    }
};

// Tables of one (precision, dimension, materials): fluids, solids and solids
// with plastic-strain planes (3-D solids are not built).
template <class R, int DIM, int NMAT>
const Ops *select_ops_nmat(int solid)
{
    // a stage tile must fit the 227 KB of shared memory a CTA may have (the
    // 3-D FP64 three-material fluid does not: not built)
    constexpr size_t lim = 227u * 1024u;
    if constexpr (StageSmem<R, DIM, NMAT, 0>::bytes <= lim) {
        if (!solid) return Impl<R, DIM, NMAT, 0>::ops();
    }
    if constexpr (DIM <= 2) {
        if constexpr (StageSmem<R, DIM, NMAT, 1>::bytes <= lim)
            if (solid == 1) return Impl<R, DIM, NMAT, 1>::ops();
        if constexpr (StageSmem<R, DIM, NMAT, 2>::bytes <= lim)
            if (solid == 2) return Impl<R, DIM, NMAT, 2>::ops();
    }
    return nullptr;
}

}  // namespace dfv

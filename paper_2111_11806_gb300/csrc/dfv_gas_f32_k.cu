// dfv_gas_f32_k.cu -- launchers of the single-gas FP32 stage kernels: 2-D
// (dfv_gasw.cuh) and 3-D (dfv_gas3.cuh), and the TMA tensor maps the 3-D
// kernel reads its plane boxes through.  Built with the fast single-precision
// divide and square root and flush-to-zero, like the other FP32 kernels.
#include <cstring>

#include <cudaTypedefs.h>

#include "dfv_gas3.cuh"
#include "dfv_gasw.cuh"

namespace dfv {

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links the runtime only)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

}  // namespace

int gasw_max_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gasw_stage<3>, GaswT::THREADS, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

cudaError_t gasw_stage(int stage, const GaswArgs &a, int grid, cudaStream_t st)
{
    const dim3 g(grid < 1 ? 1 : grid), b(GaswT::THREADS);
    if (stage == 1) return launch_pdl(k_gasw_stage<1>, g, b, 0, st, a);
    if (stage == 2) return launch_pdl(k_gasw_stage<2>, g, b, 0, st, a);
    return launch_pdl(k_gasw_stage<3>, g, b, 0, st, a);
}

int gasw_rows(long long cells)
{
    // measured on the cylinders and the 256-ellipse batch: 4-row chunks
    // below 2^19 cells (512^2: 5.7e9 against 5.2e9 cell-updates/s at 8
    // rows), then 8, growing to at most 32 while at least four items remain
    // per resident warp (152 SMs x 20 warps); 64-row chunks were 2 % slower
    // than 32 on the batch
    const long long target = 4LL * 152 * GaswT::MIN_CTAS * GaswT::WARPS;
    int rows = cells < (1LL << 19) ? 4 : 8;
    while (rows < 32 && cells / ((long long)GaswT::OWN * rows * 2) >= target) rows *= 2;
    return rows;
}

cudaError_t gas3_prepare()
{
    const int bytes = (int)sizeof(Gas3Smem);
    cudaError_t e = cudaSuccess;
    const void *k[6] = {(const void *)k_gas3_stage<1, true>,  (const void *)k_gas3_stage<2, true>,
                        (const void *)k_gas3_stage<3, true>,  (const void *)k_gas3_stage<1, false>,
                        (const void *)k_gas3_stage<2, false>, (const void *)k_gas3_stage<3, false>};
    for (int i = 0; i < 6 && e == cudaSuccess; i++)
        e = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

bool gas3_encode_map(CUtensorMap *map, const void *base, int n0, int n1, int n2, long long pitch)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || n0 % 4 != 0 || pitch % 4 != 0 || ((uintptr_t)base & 15u) != 0) return false;
    using T = Gas3T;
    const cuuint64_t dims[4] = {(cuuint64_t)n0, (cuuint64_t)n1, (cuuint64_t)n2, (cuuint64_t)T::BV};
    const cuuint64_t strides[3] = {(cuuint64_t)n0 * 4u, (cuuint64_t)n0 * (cuuint64_t)n1 * 4u, (cuuint64_t)pitch * 4u};
    const cuuint32_t box[4] = {(cuuint32_t)T::BX, (cuuint32_t)T::BY, 1u, (cuuint32_t)T::BV};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t gas3_stage(int stage, const Gas3Args &a, const CUtensorMap *map, cudaStream_t st)
{
    const dim3 g((a.n0 + Gas3T::TX - 1) / Gas3T::TX, (a.n1 + Gas3T::TY - 1) / Gas3T::TY, (a.n2 + a.zc - 1) / a.zc);
    const dim3 b(Gas3T::THREADS);
    const size_t sm = sizeof(Gas3Smem);
    if (map) {
        const CUtensorMap m = *map;
        if (stage == 1) return launch_pdl(k_gas3_stage<1, true>, g, b, sm, st, a, m);
        if (stage == 2) return launch_pdl(k_gas3_stage<2, true>, g, b, sm, st, a, m);
        return launch_pdl(k_gas3_stage<3, true>, g, b, sm, st, a, m);
    }
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    if (stage == 1) return launch_pdl(k_gas3_stage<1, false>, g, b, sm, st, a, none);
    if (stage == 2) return launch_pdl(k_gas3_stage<2, false>, g, b, sm, st, a, none);
    return launch_pdl(k_gas3_stage<3, false>, g, b, sm, st, a, none);
}

}  // namespace dfv

// dfv_gas_f32_k.cu -- launchers of the 2-D single-gas FP32 stage kernel
// (dfv_gas.cuh) and the TMA tensor maps it reads its tiles through.  Built
// with the fast single-precision divide and square root, like the other FP32
// kernels.
#include <cudaTypedefs.h>

#include "dfv_gas.cuh"
#include "dfv_gas3.cuh"
#include "dfv_gasw.cuh"

namespace dfv {

namespace {

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

cudaError_t gas_prepare()
{
    const int bytes = (int)sizeof(GasSmem);
    cudaError_t e = cudaFuncSetAttribute(k_gas_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gas_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gas_stage<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

int gas_max_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gas_stage<3>, GasT::THREADS, sizeof(GasSmem)) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

cudaError_t gas_stage(int stage, const GasArgs &a, int grid, cudaStream_t st)
{
    const dim3 g(grid < 1 ? 1 : grid), b(GasT::THREADS);
    const size_t sm = sizeof(GasSmem);
    if (stage == 1) return launch_pdl(k_gas_stage<1>, g, b, sm, st, a);
    if (stage == 2) return launch_pdl(k_gas_stage<2>, g, b, sm, st, a);
    return launch_pdl(k_gas_stage<3>, g, b, sm, st, a);
}

bool gas_encode_maps(CUtensorMap maps[GasT::NMAP], const void *const bases[3], long long off, int n0, int n1,
                     long long pitch)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || n0 % 4 != 0 || pitch % 4 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n0, (cuuint64_t)n1, (cuuint64_t)GasT::NP};
    const cuuint64_t strides[2] = {(cuuint64_t)n0 * 4u, (cuuint64_t)pitch * 4u};
    const cuuint32_t halo_box[3] = {(cuuint32_t)GasT::BX, (cuuint32_t)GasT::BY, (cuuint32_t)GasT::NP};
    const cuuint32_t own_box[3] = {(cuuint32_t)GasT::TX, (cuuint32_t)GasT::TY, (cuuint32_t)GasT::NP};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int k = 0; k < GasT::NMAP; k++) {
        void *base = (char *)const_cast<void *>(bases[k < 3 ? k : 0]) + 4 * off;
        if (((uintptr_t)base & 15u) != 0) return false;
        const CUresult r = fn(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                              k < 3 ? halo_box : own_box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

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
    // about 14,600 items of 28 columns (four per resident warp of 152 SMs at
    // 24 warps) before the chunks grow past 8 rows
    const long long target = 4LL * 152 * 24;
    int rows = 8;
    while (rows < 64 && cells / (28LL * rows * 2) >= target) rows *= 2;
    return rows;
}

cudaError_t gas3_prepare()
{
    const int bytes = (int)sizeof(Gas3Smem);
    cudaError_t e = cudaFuncSetAttribute(k_gas3_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gas3_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gas3_stage<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t gas3_stage(int stage, const Gas3Args &a, cudaStream_t st)
{
    const dim3 g((a.n0 + Gas3T::TX - 1) / Gas3T::TX, (a.n1 + Gas3T::TY - 1) / Gas3T::TY, (a.n2 + a.zc - 1) / a.zc);
    const dim3 b(Gas3T::THREADS);
    const size_t sm = sizeof(Gas3Smem);
    if (stage == 1) return launch_pdl(k_gas3_stage<1>, g, b, sm, st, a);
    if (stage == 2) return launch_pdl(k_gas3_stage<2>, g, b, sm, st, a);
    return launch_pdl(k_gas3_stage<3>, g, b, sm, st, a);
}

}  // namespace dfv

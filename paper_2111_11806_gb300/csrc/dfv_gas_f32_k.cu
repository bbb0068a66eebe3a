// dfv_gas_f32_k.cu -- launchers of the single-gas FP32 stage kernels: 2-D
// (dfv_gasw.cuh) and 3-D (dfv_gas3.cuh).  Built with the fast single-precision
// divide and square root and flush-to-zero, like the other FP32 kernels.
#include "dfv_gas3.cuh"
#include "dfv_gasw.cuh"

namespace dfv {

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

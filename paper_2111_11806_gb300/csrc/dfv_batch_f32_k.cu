// Batch kernels of the FP32 form.
#include "dfv_batch.cuh"

namespace dfv {
Kern batch_kernels_f32(int nmat) { return batch_kernels<float>(nmat); }
}  // namespace dfv

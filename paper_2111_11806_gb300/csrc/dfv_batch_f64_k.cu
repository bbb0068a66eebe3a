// Batch kernels of the plain FP64 form.
#include "dfv_batch.cuh"

namespace dfv {
Kern batch_kernels_f64(int nmat) { return batch_kernels<double>(nmat); }
}  // namespace dfv

// One launcher table of the CUDA path: precision DFV_TU_REAL, dimension
// DFV_TU_DIM and DFV_TU_NMAT materials, every solid kind that is built.  The
// build compiles this file once per combination (defines set by _build.py)
// so that the kernels compile in parallel.
#include "dfv_inst.cuh"

#if !defined(DFV_TU_REAL) || !defined(DFV_TU_DIM) || !defined(DFV_TU_NMAT) || !defined(DFV_TU_NAME)
#error "dfv_inst_tu.cu is compiled once per (precision, dimension, materials) with DFV_TU_* defines"
#endif

namespace dfv {
const Ops *DFV_TU_NAME(int solid) { return select_ops_nmat<DFV_TU_REAL, DFV_TU_DIM, DFV_TU_NMAT>(solid); }
}  // namespace dfv

// Launcher tables of the f64 form, 1-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f64_d1(int nmat, int solid) { return select_ops_dim<double, 1>(nmat, solid); }
}  // namespace dfv

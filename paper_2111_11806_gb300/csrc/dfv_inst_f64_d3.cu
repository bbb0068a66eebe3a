// Launcher tables of the f64 form, 3-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f64_d3(int nmat, int solid) { return select_ops_dim<double, 3>(nmat, solid); }
}  // namespace dfv

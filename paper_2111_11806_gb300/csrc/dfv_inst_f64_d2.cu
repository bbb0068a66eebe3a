// Launcher tables of the f64 form, 2-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f64_d2(int nmat, int solid) { return select_ops_dim<double, 2>(nmat, solid); }
}  // namespace dfv

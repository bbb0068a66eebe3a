// Launcher tables of the f32 form, 3-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f32_d3(int nmat, int solid) { return select_ops_dim<float, 3>(nmat, solid); }
}  // namespace dfv

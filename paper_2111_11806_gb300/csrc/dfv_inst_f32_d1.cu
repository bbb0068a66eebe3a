// Launcher tables of the f32 form, 1-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f32_d1(int nmat, int solid) { return select_ops_dim<float, 1>(nmat, solid); }
}  // namespace dfv

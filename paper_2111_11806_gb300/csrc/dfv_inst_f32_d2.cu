// Launcher tables of the f32 form, 2-D.
#include "dfv_inst.cuh"

namespace dfv {
const Ops *ops_f32_d2(int nmat, int solid) { return select_ops_dim<float, 2>(nmat, solid); }
}  // namespace dfv

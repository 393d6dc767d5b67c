// Step kernels with float storage, whole-row ring variants (one translation unit per storage type
// and ring kind, compiled in parallel).
#include "lb_step.cuh"

namespace lbm {

LB_STEP_UNIT(f32, float, 0)

}  // namespace lbm

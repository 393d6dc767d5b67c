// Step kernels with double storage, stage ring variants (one translation unit per storage type
// and ring kind, compiled in parallel).
#include "lb_step.cuh"

namespace lbm {

LB_STEP_UNIT(f64, double, 1)

}  // namespace lbm

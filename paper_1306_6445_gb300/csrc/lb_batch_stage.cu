// Batched step kernels with the stage ring (FP32, FP64), compiled apart from the
// whole-row ring ones of lb_batch_kernels.cu.
#include "lb_step.cuh"

namespace lbm {

LB_BATCH_UNIT(f32, float, 1)
LB_BATCH_UNIT(f64, double, 1)

}  // namespace lbm

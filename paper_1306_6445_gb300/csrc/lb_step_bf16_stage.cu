// Step kernels with __nv_bfloat16 storage, stage ring variants (one translation unit per storage type
// and ring kind, compiled in parallel).
#include "lb_step.cuh"

namespace lbm {

LB_STEP_UNIT(bf16, __nv_bfloat16, 1)

}  // namespace lbm

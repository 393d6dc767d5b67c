// Step kernels with double storage (one translation unit per precision, compiled in parallel).
#include "lb_step.cuh"

namespace lbm {

cudaError_t step_f64(const Consts &c, const Geom &g, const StepLaunch &l, int order,
                      const void *tensor_map_in, void *gout, int *err, cudaStream_t st,
                      bool configure) {
    return step_dispatch<double>(c, g, l, order, *static_cast<const CUtensorMap *>(tensor_map_in),
                              gout, err, st, configure);
}

int occupancy_f64(int variant, int eos_kind, int bc) {
    return occupancy<double>(variant, eos_kind, bc);
}

}  // namespace lbm

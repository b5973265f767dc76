// Fused FP32 lower-level solve: instantiations for scenes with a road profile
// (curvature and lane limits evaluated per timestep; fused_kernel.cuh).
#include "fused_kernel.cuh"

namespace plan {

void fused_setup_road() { setup_road<true>(); }

cudaError_t launch_fused_f32_road(const FusedLaunch& L, const Consts& c, const Params& prm,
                                  cudaStream_t s) {
  return launch_road<true>(L, c, prm, s);
}

}  // namespace plan

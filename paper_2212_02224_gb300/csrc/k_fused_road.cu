// Fused FP32 lower-level solve: instantiations for scenes with a road profile
// (curvature and lane limits evaluated per timestep; fused_kernel.cuh).
#include "fused_kernel.cuh"

namespace plan {

void fused_setup_road() { setup_road<true>(); }

cudaError_t launch_fused_f32_road(const DevScene* scenes, const Layout* layout, const double* obs,
                                  const Tile* tiles, int n_tiles, int wps, int spc, const double* p,
                                  const Consts& c, const Params& prm, double* xi, double* r,
                                  double* cu, int* st, cudaStream_t s) {
  return launch_road<true>(scenes, layout, obs, tiles, n_tiles, wps, spc, p, c, prm, xi, r, cu, st, s);
}

}  // namespace plan

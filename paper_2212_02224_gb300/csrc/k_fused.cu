// Fused FP32 lower-level solve: host side of the scenes without a road profile
// (the kernel template is in fused_kernel.cuh; road-profile instantiations in
// k_fused_road.cu).
#include "fused_kernel.cuh"

namespace plan {

void fused_setup() {
  setup_road<false>();
  fused_setup_road();
}

bool fused_supported(int n, int m) {
  return (n == 8 || n == 11 || n == 16) && m >= 2 && m <= 256;
}

bool fused_shape_ok(int wps, int spc) {
  if (wps == 1) return spc >= 1 && spc <= 8;
  if (wps == 2) return spc == 1 || spc == 2 || spc == 4;
  return wps == 4 && spc == 1;
}

cudaError_t launch_fused_f32(const DevScene* scenes, const Layout* layout, const double* obs,
                             const Tile* tiles, int n_tiles, int wps, int spc, const double* p,
                             const Consts& c, const Params& prm, double* xi, double* r,
                             double* cu, int* st, bool road, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  if (!fused_shape_ok(wps, spc)) return cudaErrorInvalidValue;
  if (road)
    return launch_fused_f32_road(scenes, layout, obs, tiles, n_tiles, wps, spc, p, c, prm, xi, r,
                                 cu, st, s);
  return launch_road<false>(scenes, layout, obs, tiles, n_tiles, wps, spc, p, c, prm, xi, r, cu, st, s);
}

}  // namespace plan

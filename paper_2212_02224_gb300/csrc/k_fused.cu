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

cudaError_t launch_fused_f32(const FusedLaunch& L, const Consts& c, const Params& prm,
                             cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  if (!fused_shape_ok(L.wps, L.spc)) return cudaErrorInvalidValue;
  if (L.persist != PLAN_PERSIST_AUTO && L.persist != PLAN_PERSIST_OFF &&
      L.persist != PLAN_PERSIST_ON)
    return cudaErrorInvalidValue;
  if (L.persist != PLAN_PERSIST_OFF && (!L.work || !L.sample_scene || L.sms < 1))
    return cudaErrorInvalidValue;
  if (L.road) return launch_fused_f32_road(L, c, prm, s);
  return launch_road<false>(L, c, prm, s);
}

}  // namespace plan

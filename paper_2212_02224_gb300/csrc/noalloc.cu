// plan_solve_fp64_noalloc: the float64 lower-level solve without any device
// allocation.  Everything the solve needs beyond the caller's inputs and
// outputs -- scene copy, basis, KKT inverses and the float64 path's
// per-iteration intermediates -- lives in one file-scope __device__ array of
// fixed size.  It exists for callers that must not allocate (see plan.h).
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "plan.h"
#include "internal.cuh"

namespace plan {

// Limits of the allocation-free entry point.
constexpr int kNaMaxB = 256;      // samples per call
constexpr int kNaMaxM = 128;      // timesteps
constexpr int kNaMaxObs = 32;     // obstacles
constexpr int kNaMaxN = kMaxCoef; // coefficients per axis
constexpr int kNaMaxSeg = 4;
constexpr int kNaMaxNe = 5;       // equality rows per axis (with goal entries)

namespace {

constexpr size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// byte sizes of the regions, at the limits
constexpr size_t kScene = al(sizeof(DevScene));
constexpr size_t kObs = al(sizeof(double) * 6 * kNaMaxObs);
constexpr size_t kLayout = al(sizeof(Layout));
constexpr size_t kSampleScene = al(sizeof(int) * kNaMaxB);
constexpr size_t kBasis64 = al(sizeof(double) * 3 * kNaMaxM * kNaMaxN);
constexpr size_t kBasis32 = al(sizeof(float) * kNaMaxM * basis32_stride(kNaMaxN));
constexpr size_t kS1_64 = al(sizeof(double) * 2 * kNaMaxN * (kNaMaxSeg + kNaMaxNe));
constexpr size_t kS1_32 = al(sizeof(float) * 2 * kNaMaxN * (kNaMaxSeg + kNaMaxNe));
constexpr size_t kPj64 = al(sizeof(double) * (kNaMaxObs + 1) * 2 * kNaMaxN * (2 * kNaMaxN + kNaMaxNe));
constexpr size_t kPj32 = al(sizeof(float) * (kNaMaxObs + 1) * 2 * kNaMaxN * (2 * kNaMaxN + kNaMaxNe));
constexpr size_t kVec = al(sizeof(double) * kNaMaxB * 32);
constexpr size_t kState = al(sizeof(double) * kNaMaxB * 6 * kNaMaxM);
constexpr size_t kEps = al(sizeof(double) * kNaMaxB * 7 * kNaMaxM);
constexpr size_t kDa = al(sizeof(double) * kNaMaxB * kNaMaxM);
constexpr size_t kScratchBytes = kScene + kObs + kLayout + kSampleScene + kBasis64 + kBasis32 +
                                 kS1_64 + kS1_32 + kPj64 + kPj32 + 4 * kVec + kState + kEps +
                                 2 * kDa;

// The scratch array (about 4.7 MB); every GPU that loads the library holds it
// until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once per device.
std::mutex g_mu;
void* g_addr[64] = {nullptr};

struct SceneParam {
  DevScene sc;
  double obs[6 * kNaMaxObs];
  int B;
};

// Writes the scene, its layout and the sample-to-scene map into the scratch.
__global__ void setup_kernel(SceneParam sp, DevScene* sc, double* obs, Layout* layout,
                             int* sample_scene) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *sc = sp.sc;
    *layout = Layout{sp.B, 0};
  }
  if (i < 6 * sp.sc.n_obs) obs[i] = sp.obs[i];
  if (i < sp.B) sample_scene[i] = 0;
}

int na_fail(int code, const char* msg) {
  set_unbound_error(msg);   // read back with plan_last_error(NULL, ...)
  return code;
}

}  // namespace
}  // namespace plan

using namespace plan;

extern "C" int plan_solve_fp64_noalloc(const plan_config* cfg, const plan_scene* scene,
                                       const double* p, int B, double* xi, double* resid,
                                       double* cu, void* stream) {
  if (!cfg || !scene) return na_fail(PLAN_EINVAL, "cfg and scene must be non-NULL");
  if (B < 0) return na_fail(PLAN_EINVAL, "B < 0");
  if (B > kNaMaxB) return na_fail(PLAN_ECAPACITY, "B exceeds 256 samples");
  if (cfg->m > kNaMaxM) return na_fail(PLAN_ECAPACITY, "m must be in [8, 128]");
  // the same checks of the lower-level parameters and of the scene as plan_init
  // and plan_solve make
  if (const char* why = lower_config_invalid(*cfg)) return na_fail(PLAN_EINVAL, why);
  if (scene->n_obs > kNaMaxObs) return na_fail(PLAN_ECAPACITY, "n_obs must be in [0, 32]");
  if (const char* why = scene_invalid(*scene, cfg->lane_margin)) return na_fail(PLAN_EINVAL, why);
  if (B == 0) return PLAN_OK;
  if (!p || !resid || !cu) return na_fail(PLAN_EINVAL, "p, resid and cu must be non-NULL");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return na_fail(PLAN_ECUDA, "no current CUDA device");
  }
  unsigned char* base = nullptr;
  {
    // first call on this device: look up the array's device address (with
    // this device current); host code must not use g_scratch's own address
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return na_fail(PLAN_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char* q = base + off; off += bytes; return q; };
  DevScene* d_sc = reinterpret_cast<DevScene*>(take(kScene));
  double* d_obs = reinterpret_cast<double*>(take(kObs));
  Layout* d_lay = reinterpret_cast<Layout*>(take(kLayout));
  int* d_ss = reinterpret_cast<int*>(take(kSampleScene));
  Consts c{};
  c.basis64 = reinterpret_cast<double*>(take(kBasis64));
  c.basis32 = reinterpret_cast<float*>(take(kBasis32));
  c.s1_64 = reinterpret_cast<double*>(take(kS1_64));
  c.s1_32 = reinterpret_cast<float*>(take(kS1_32));
  c.pj64 = reinterpret_cast<double*>(take(kPj64));
  c.pj32 = reinterpret_cast<float*>(take(kPj32));
  c.m = cfg->m;
  c.n = cfg->n_coef;
  c.n_seg = cfg->n_seg;
  c.max_obs = scene->n_obs;
  c.goal = cfg->goal;
  c.ne = 3 + 2 * cfg->goal;
  Plain64Work w{};
  w.xibarp = reinterpret_cast<double*>(take(kVec));
  w.xi = reinterpret_cast<double*>(take(kVec));
  w.lam = reinterpret_cast<double*>(take(kVec));
  w.w = reinterpret_cast<double*>(take(kVec));
  w.state = reinterpret_cast<double*>(take(kState));
  w.eps = reinterpret_cast<double*>(take(kEps));
  w.da = reinterpret_cast<double*>(take(kDa));
  w.xprev = reinterpret_cast<double*>(take(kDa));

  Params prm{};
  prm.m = cfg->m; prm.n = cfg->n_coef; prm.n_seg = cfg->n_seg; prm.K = cfg->inner_iters;
  prm.L = 1; prm.d_p = 2 * cfg->n_seg + 2 * cfg->goal; prm.max_obs = scene->n_obs;
  prm.goal = cfg->goal;
  prm.dt = cfg->dt; prm.rho = cfg->rho; prm.kp_lat = cfg->kp_lat; prm.kv_lat = cfg->kv_lat;
  prm.kp_lon = cfg->kp_lon; prm.v_min = cfg->v_min; prm.v_max = cfg->v_max;
  prm.a_max = cfg->a_max; prm.kappa_max = cfg->kappa_max; prm.c_max = cfg->c_max;
  prm.lane_margin = cfg->lane_margin;

  SceneParam sp{};
  const plan_ego& e = scene->ego;
  sp.sc.ego[0] = e.x; sp.sc.ego[1] = e.y; sp.sc.ego[2] = e.vx;
  sp.sc.ego[3] = e.vy; sp.sc.ego[4] = e.ax; sp.sc.ego[5] = e.ay;
  sp.sc.y_lb = cfg->lane_margin;
  sp.sc.y_ub = scene->n_lanes * scene->lane_width - cfg->lane_margin;
  sp.sc.kappa_road = scene->kappa_road;
  sp.sc.lane_width = scene->lane_width;
  sp.sc.n_lanes = scene->n_lanes;
  sp.sc.n_obs = scene->n_obs;
  sp.sc.obs_off = 0;
  fill_road(sp.sc, *scene, cfg->lane_margin);
  for (int i = 0; i < scene->n_obs; ++i) {
    const plan_obstacle& o = scene->obs[i];
    const double v[6] = {o.x0, o.y0, o.vx, o.vy, o.a, o.b};
    for (int k = 0; k < 6; ++k) sp.obs[6 * i + k] = v[k];
  }
  sp.B = B;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nthr = std::max(B, 6 * kNaMaxObs);
  setup_kernel<<<(nthr + 127) / 128, 128, 0, s>>>(sp, d_sc, d_obs, d_lay, d_ss);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = build_constants(c, prm, s);
  if (err == cudaSuccess)
    err = launch_plain64(d_sc, d_lay, d_ss, d_obs, B, p, c, prm, w, xi, resid, cu, nullptr, s);
  if (err != cudaSuccess) return na_fail(PLAN_ECUDA, cudaGetErrorString(err));
  return PLAN_OK;
}

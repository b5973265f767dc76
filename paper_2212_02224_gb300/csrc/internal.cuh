// Internal declarations of the planner library (device structs, launchers).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace plan {

constexpr int kMaxCoef = 16;     // coefficients per axis
constexpr int kMaxDp = PLAN_MAX_DP;   // entries of p (4 + 4 set-points, 2 goal entries)
constexpr int kMaxObs = 64;      // obstacles per scene
constexpr int kMaxM = 256;       // timesteps
constexpr int kMaxEliteC = 2048; // ConstraintEliteSet size
constexpr int kMaxRoad = 8;      // knots of a road profile

// Geometry of one scene as the kernels see it.
struct DevScene {
  double ego[6];        // b0: x, y, vx, vy, ax, ay
  double y_lb, y_ub;    // lane-boundary rows of Table I (no road profile)
  double kappa_road;    // road curvature (centripetal bound, no road profile)
  double lane_width;
  int n_lanes, n_obs;
  int obs_off;          // first obstacle in the obstacle array (6 doubles each)
  int n_road;           // knots of the road profile (0: constant road)
  // road profile in the scene's frame (knot s already shifted by the origin),
  // edges already moved inwards by the lane margin: {s, kappa, y_lb, y_ub}
  double road[kMaxRoad][4];
};

// The road profile of a scene in the scene's frame, edges moved inwards by the
// lane margin (host side; the knots are validated by the caller).
inline void fill_road(DevScene& d, const plan_scene& s, double lane_margin) {
  d.n_road = s.n_road;
  for (int i = 0; i < s.n_road && i < kMaxRoad; ++i) {
    d.road[i][0] = s.road[i].s - s.road_origin;
    d.road[i][1] = s.road[i].kappa;
    d.road[i][2] = s.road[i].lb + lane_margin;
    d.road[i][3] = s.road[i].ub - lane_margin;
  }
}

// Road knots of a scene: NULL message when valid, else the reason.
inline const char* road_invalid(const plan_scene& s, double lane_margin) {
  if (s.n_road < 0 || s.n_road > kMaxRoad) return "n_road must be in [0, 8]";
  if (s.n_road > 0 && !s.road) return "road is NULL";
  if (!(s.road_origin == s.road_origin) || s.road_origin - s.road_origin != 0.0)
    return "road_origin is not finite";
  for (int i = 0; i < s.n_road; ++i) {
    const plan_road_knot& k = s.road[i];
    const double v[4] = {k.s, k.kappa, k.lb, k.ub};
    for (double x : v)
      if (x - x != 0.0) return "road knot not finite";
    if (i > 0 && !(k.s > s.road[i - 1].s)) return "road knots: s must increase";
    if (!(k.ub - k.lb - 2 * lane_margin > 0)) return "road knot narrower than twice lane_margin";
  }
  return nullptr;
}

// The parameters of cfg that the lower-level solve uses: NULL when valid, else
// the reason (host side; shared by every entry point that takes a config).
inline const char* lower_config_invalid(const plan_config& c) {
  if (c.m < 8 || c.m > kMaxM) return "m must be in [8, 256]";
  if (c.n_coef < 4 || c.n_coef > kMaxCoef) return "n_coef must be in [4, 16]";
  if (c.n_seg < 1 || c.n_seg > 4 || c.n_seg > c.m) return "n_seg must be in [1, 4]";
  if (c.goal != 0 && c.goal != 1) return "goal must be 0 or 1";
  if (c.goal && c.n_coef < 6) return "goal entries need n_coef >= 6 (five equality rows on the y axis)";
  if (c.inner_iters < 1) return "inner_iters must be >= 1";
  if (!(c.dt > 0) || !(c.rho > 0) || !std::isfinite(c.dt) || !std::isfinite(c.rho))
    return "dt and rho must be finite and > 0";
  if (!std::isfinite(c.kp_lat) || !std::isfinite(c.kv_lat) || !std::isfinite(c.kp_lon))
    return "the tracking gains must be finite";
  if (!(c.v_min >= 0) || !(c.v_max > c.v_min) || !std::isfinite(c.v_max))
    return "need 0 <= v_min < v_max (finite)";
  if (!(c.a_max > 0) || !(c.kappa_max > 0) || !(c.c_max > 0) || !std::isfinite(c.a_max) ||
      !std::isfinite(c.kappa_max) || !std::isfinite(c.c_max))
    return "a_max, kappa_max, c_max must be finite and > 0";
  if (!(c.lane_margin >= 0) || !std::isfinite(c.lane_margin)) return "lane_margin must be >= 0";
  return nullptr;
}

// A scene's geometry: NULL when valid, else the reason (host side; the
// obstacle capacity is the caller's check).
inline const char* scene_invalid(const plan_scene& s, double lane_margin) {
  if (s.n_lanes < 1) return "n_lanes must be >= 1";
  if (!(s.lane_width > 0) || !std::isfinite(s.lane_width)) return "lane_width must be > 0";
  if (!(s.n_lanes * s.lane_width - 2 * lane_margin > 0)) return "road narrower than twice lane_margin";
  if (s.n_obs < 0) return "n_obs < 0";
  if (s.n_obs > 0 && !s.obs) return "obs is NULL";
  const double* e = &s.ego.x;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(e[i])) return "ego state not finite";
  if (!std::isfinite(s.kappa_road)) return "kappa_road not finite";
  for (int i = 0; i < s.n_obs; ++i) {
    const plan_obstacle& o = s.obs[i];
    if (!(o.a > 0) || !(o.b > 0) || !std::isfinite(o.a) || !std::isfinite(o.b) ||
        !std::isfinite(o.x0) || !std::isfinite(o.y0) || !std::isfinite(o.vx) || !std::isfinite(o.vy))
      return "obstacle invalid (finite entries, axes > 0)";
  }
  return road_invalid(s, lane_margin);
}

// Road curvature and lane limits at x (linear between knots, constant beyond).
template <class T>
__host__ __device__ inline void road_eval(const DevScene& sc, T x, T* kappa, T* ylb, T* yub) {
  const int n = sc.n_road;
  if (n == 0) {
    *kappa = T(sc.kappa_road); *ylb = T(sc.y_lb); *yub = T(sc.y_ub);
    return;
  }
  if (!(x > T(sc.road[0][0]))) {
    *kappa = T(sc.road[0][1]); *ylb = T(sc.road[0][2]); *yub = T(sc.road[0][3]);
    return;
  }
  int i = 0;
  while (i + 1 < n && T(sc.road[i + 1][0]) < x) ++i;
  if (i + 1 >= n) {
    *kappa = T(sc.road[n - 1][1]); *ylb = T(sc.road[n - 1][2]); *yub = T(sc.road[n - 1][3]);
    return;
  }
  const T s0 = T(sc.road[i][0]), s1 = T(sc.road[i + 1][0]);
  const T w = (x - s0) / (s1 - s0);
  *kappa = T(sc.road[i][1]) + w * (T(sc.road[i + 1][1]) - T(sc.road[i][1]));
  *ylb = T(sc.road[i][2]) + w * (T(sc.road[i + 1][2]) - T(sc.road[i][2]));
  *yub = T(sc.road[i][3]) + w * (T(sc.road[i + 1][3]) - T(sc.road[i][3]));
}

// Per-scene state of the outer loop (Alg. 1), device resident.
struct DevCem {
  double mu[kMaxDp];
  double sigma[kMaxDp * kMaxDp];   // leading dimension kMaxDp
  double chol[kMaxDp * kMaxDp];    // lower Cholesky factor of sigma + eps I
  double best_p[kMaxDp];
  double best_xi[2 * kMaxCoef];
  double best_cost, best_r, best_cu;
  unsigned long long seed, step;
  int fresh, best_index;
  int pad[2];
};

// Numeric parameters (plan_config) for the kernels.
struct Params {
  int m, n, n_seg, K;
  int L, n_c, q, d_p;
  int max_obs, goal;   // goal: p ends with x_f, y_f (Eq. final_boundary rows)
  double dt, rho, kp_lat, kv_lat, kp_lon, gamma, eta, cov_eps;
  double v_min, v_max, a_max, kappa_max, c_max, lane_margin, v_des_lo, v_des_hi;
};

// Constants built in float64 on the device by build_constants().
//   basis64 [3][m][n]  W, Wd, Wdd row-major (FP64 path)
//   basis32 [m][stride] per timestep the rows W[t], Wd[t], Wdd[t], each padded
//           to ncp = 4 ceil(n / 4) floats, row stride basis32_stride(n) floats
//           (an odd multiple of 4, so 16-byte loads of 8 consecutive t are
//           free of shared-memory bank conflicts)
//   s1_*    [2][n][n_seg + ne]  Step-1 maps: xi_bar_axis = Gs p_axis + Hs b_axis
//   pj_*    [N + 1][2][n][2n + ne]  per obstacle count N and axis, row k:
//           M[k][:], MP[k][:], C[k][:] with xi = M r + C b (KKT inverse of
//           the xi-step) and MP = rho M P, P = F^T F + G^T G of that axis.
// b of an axis (the columns of Hs and C): the initial rows (position,
// velocity, acceleration at t0) and, with goal entries, the final rows of
// Eq. final_boundary: x(t_f) on the x axis; y(t_f), ydot(t_f) on the y axis.
// ne = 3 without goal entries, 5 with them (the x axis leaves column 4 zero).
struct Consts {
  double* basis64;
  float* basis32;
  double* s1_64;
  float* s1_32;
  double* pj64;
  float* pj32;
  int m, n, n_seg, max_obs;
  int ne, goal;
};

// Equality rows per axis: 3 initial rows, plus 1 (x) or 2 (y) final rows.
__host__ __device__ constexpr int eq_rows(int axis, int goal) {
  return 3 + (goal ? (axis == 0 ? 1 : 2) : 0);
}

// Layout of one call: scene s owns samples [off, off + B).
struct Layout {
  int B, off;
};

// A tile of the fused kernel: `count` samples of `scene` starting at `first`
// (scene-relative).
struct Tile {
  int scene, first, count, pad;
};

__host__ __device__ constexpr int basis32_ncp(int n) { return (n + 3) / 4 * 4; }
__host__ __device__ constexpr int basis32_stride(int n) {
  return ((3 * basis32_ncp(n)) / 4) % 2 == 1 ? 3 * basis32_ncp(n) : 3 * basis32_ncp(n) + 4;
}

// Programmatic dependent launch within the MPC cycle (sample -> solve ->
// select): a kernel launched with launch_pdl may start while its predecessor
// in the stream finishes; it must call pdl_wait() before touching anything the
// predecessor writes or reads, and calls pdl_trigger() once its successor may
// be scheduled (only after its own wait, or at the end of its main work, so
// that waiting grids never hold resources an unfinished earlier grid needs).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Launchers (return the cudaError_t of the launch).
cudaError_t build_constants(const Consts& c, const Params& p, cudaStream_t s);

bool fused_supported(int n, int m);
// wps = warps per sample (1, 2, 4), spc = samples per CTA (spc * wps <= 8)
bool fused_shape_ok(int wps, int spc);

// One launch of the fused FP32 solve over `total` samples of the scenes.
struct FusedLaunch {
  const DevScene* scenes;
  const Layout* layout;
  const double* obs;
  const Tile* tiles;        // tiles of spc samples (one CTA each)
  int n_tiles;
  const int* sample_scene;  // scene of every sample (persistent form)
  int total;
  int* work;                // two zeroed ints owned by the context (persistent form)
  int sms;
  int persist;              // PLAN_PERSIST_AUTO, _OFF or _ON
  int wps, spc;
  bool road;                // some scene has a road profile (selects the instantiations
                            // that evaluate curvature and lane limits per timestep)
  const double* p;
  double *xi, *r, *cu;
  int* st;
};
cudaError_t launch_fused_f32(const FusedLaunch& L, const Consts& c, const Params& prm,
                             cudaStream_t s);

// Tensor-core modes (PLAN_PREC_TF32, _BF16, _TF32X3): tiles of
// tc_samples_per_cta() samples; err is set to 1 if a wait timed out.
bool tc_supported(int n, int m, int max_obs);
void tc_setup();
int tc_samples_per_cta();
cudaError_t launch_tc(int prec, const DevScene* scenes, const Layout* layout, const double* obs,
                      const Tile* tiles, int n_tiles, const double* p, const Consts& c,
                      const Params& prm, double* xi, double* r, double* cu, int* st, int* err,
                      cudaStream_t s);
// One bounded mbarrier wait that receives no arrival (k_tc.cu): *timed_out = 1
// when it gave up after `limit` SM cycles.  Synchronous on s.
cudaError_t wait_probe(long long limit, cudaStream_t s, int* timed_out);
// SM cycles per iteration of the wide-N tensor-core contractions, per CTA
// (5 doubles each); see plan_probe_tc_wide.
cudaError_t tc_wide_probe(int passes, int iters, int ctas, double* cycles, cudaStream_t s,
                          int* timed_out);

// Arithmetic throughput probe (k_peaks.cu): out[0..4] as plan_probe_alu.
int probe_alu(double* out, cudaStream_t s);

// Differentiable Step-1 layer (k_qp.cu).
cudaError_t launch_qp_forward(const Consts& c, const double* p, const double* b0, int B,
                              double* xi, cudaStream_t s);
cudaError_t launch_qp_backward(const Consts& c, const double* g, int B, double* grad_p,
                               double* grad_b0, cudaStream_t s);

struct Plain64Work {   // HBM intermediates of the FP64 path
  double* xibarp;  // [B][32] M xi_bar + C b
  double* xi;      // [B][32]
  double* lam;     // [B][32]
  double* w;       // [B][32]
  double* state;   // [B][6][m]
  double* eps;     // [B][7][m]
  double* da;      // [B][m]
  double* xprev;   // [B][m] positions x of the previous iterate (road curvature)
};

cudaError_t launch_plain64(const DevScene* scenes, const Layout* layout, const int* sample_scene,
                           const double* obs, int total_B, const double* p, const Consts& c,
                           const Params& prm, const Plain64Work& w, double* xi_out, double* r,
                           double* cu, int* st, cudaStream_t s);

// pdl = false: a full dependency on the preceding work of the stream.  zbuf:
// the normals of iteration l written by launch_normals ([total B][d_p]), or
// NULL to draw them in the sampling kernel.
cudaError_t launch_sample(const DevScene* scenes, const Layout* layout, const DevCem* cem, int S,
                          int max_B, int l, const Params& prm, double* p, cudaStream_t s,
                          bool pdl = true, const double* zbuf = nullptr);
// The Cholesky factor of one imported sampling state (not fresh), on the
// device, by the selection kernels' routine.
cudaError_t launch_import_chol(DevCem* cem, const Params& prm, cudaStream_t s);
// The standard normals of outer iteration l >= 2 for every sample (Philox and
// Box-Muller in float64), into zbuf; a plain launch, meant for a stream that
// runs beside the solve of iteration l - 1.
cudaError_t launch_normals(const Layout* layout, const DevCem* cem, int S, int max_B, int l,
                           const Params& prm, double* zbuf, cudaStream_t s);
// Staging of one cycle through a pinned, device-mapped host buffer `io`: the
// scene record (offset 0), its obstacle rows (o_obs) and the sampling state
// (o_cem) go to the device copies; the final state and the tensor-core timeout
// flag come back to offset o_ret.  One CTA each.  The input kernel also
// factors a warm start's covariance (the selection kernels' routine).
cudaError_t launch_io_in(const void* io, size_t o_obs, size_t o_cem, DevScene* scene, double* obs,
                         DevCem* cem, const Params& prm, cudaStream_t s);
cudaError_t launch_io_out(const DevCem* cem, const int* tc_err, void* io, size_t o_ret,
                          cudaStream_t s);

cudaError_t launch_select_update(const Layout* layout, DevCem* cem, int S, int l,
                                 const Params& prm, const double* p, const double* xi,
                                 const double* r, const double* cu, int* elite_out,
                                 int max_B, cudaStream_t s);

static_assert(sizeof(DevCem) % sizeof(unsigned long long) == 0, "DevCem is copied in 8-byte words");
static_assert(sizeof(DevScene) % sizeof(unsigned long long) == 0, "DevScene is copied in 8-byte words");

cudaError_t launch_cem_copy(DevCem* dst, const DevCem* src, const int* idx, int S, bool scatter,
                            cudaStream_t s);

// Error message of a call that has no context (reported by plan_last_error(NULL)).
void set_unbound_error(const char* msg);

cudaError_t launch_select_only(const double* r, const double* cu, int B, int n_c, int q,
                               int* elite, cudaStream_t s);
cudaError_t launch_update_only(const double* p_elite, const double* cost, int q, int d_p,
                               double gamma, double eta, double* mu, double* sigma,
                               cudaStream_t s);

}  // namespace plan

struct plan_ctx;
namespace plan {
// Hooks of the serving loop into a context (plan_api.cu).
size_t ctx_bytes(const plan_ctx* ctx);
const char* ctx_error(const plan_ctx* ctx);
int ctx_make_state(plan_ctx* ctx, const plan_cem_state* st, int n_lanes, double lane_width,
                   double ego_x, DevCem* out);
// One Alg. 1 run over S scenes, launched directly (no graph) on `s`: scene
// slots, states init[s] (or table[gather[s]] where gather[s] >= 0), L outer
// iterations, then table[scatter[s]] = final state and results (pinned host,
// S entries) = final states.
int ctx_wave(plan_ctx* ctx, const plan_scene* scenes, const int* B, int S, const DevCem* init,
             const int* gather, const int* scatter, DevCem* table, DevCem* results,
             cudaStream_t s);
}  // namespace plan

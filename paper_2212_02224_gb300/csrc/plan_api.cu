// C ABI of the planner: context, device arena, staging, launch sequences and
// CUDA-graph capture of whole Alg. 1 runs.  See include/plan.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "plan.h"
#include "internal.cuh"

namespace plan {
void cem_setup();
void fused_setup();
}  // namespace plan

using namespace plan;

namespace {

// Device buffers describing one set of scenes and their sample layout.
struct SceneSet {
  DevScene* scenes = nullptr;
  double* obs = nullptr;
  Layout* layout = nullptr;
  Tile* tiles = nullptr;
  int* sample_scene = nullptr;
  bool road = false;       // some uploaded scene has a road profile
};

struct GraphEntry {
  std::vector<int> B;
  bool road = false;       // kernel variant captured (road profile or not)
  bool io = false;         // with the host-mapped staging of plan_step at head and tail
  SceneSet set;            // own layout / tiles / sample_scene (scenes+obs shared)
  cudaGraphExec_t exec = nullptr;
  int total_B = 0, max_B = 0;
};

}  // namespace

struct plan_ctx {
  plan_config cfg{};
  Params prm{};
  Consts c{};
  int device = 0;
  int sms = 0;                      // multiprocessors of the device
  int tune_wps = 0, tune_spc = 0;   // fused-kernel shape; 0 = automatic
  int persist = PLAN_PERSIST_AUTO;  // launch form of the fused kernel
  cudaStream_t internal = nullptr;
  cudaStream_t capture = nullptr;
  // side branch of the captured cycle: the next iteration's normals are drawn
  // on `side` while the current iteration solves (fork / join events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

  // arena
  std::vector<void*> allocs;
  size_t arena_bytes = 0;
  int* rows = nullptr;     // [2][max_scenes] gather / scatter rows of the serving loop
  SceneSet tr;             // transient scenes (plan_solve)
  // bytes of the last upload into `tr` (scene records, obstacle rows, layout,
  // tiles, sample-to-scene map) and an event recorded after its copies: a call
  // whose upload would write the same bytes waits on that event instead
  std::vector<unsigned char> tr_key;
  bool tr_key_ok = false;
  cudaEvent_t tr_ready = nullptr;
  SceneSet res;            // resident scene slots (plan_step_resident)
  DevCem* cem = nullptr;   // [max_scenes]
  double* p = nullptr;     // [max_samples][d_p]
  double* xi = nullptr;    // [max_samples][2n]
  double* r = nullptr;
  double* cu = nullptr;
  int* elite = nullptr;    // [max_scenes][q]
  int* tc_err = nullptr;   // timeout flag of the tensor-core kernel
  int* work = nullptr;     // [2] sample counter and finished groups of the persistent kernel
  double* zbuf = nullptr;  // [max_samples][d_p] normals of the next outer iteration
  Plain64Work pw{};
  DevCem* cem_tmp = nullptr;   // single-stage sampling
  Layout* layout_tmp = nullptr;

  // plan_step's pinned, device-mapped staging: scene record at 0, obstacle rows
  // at io_obs (max_obs rows), sampling state at io_cem, result at io_ret
  unsigned char* io = nullptr;
  void* io_dev = nullptr;
  size_t io_obs = 0, io_cem = 0, io_ret = 0;

  // pinned staging
  unsigned char* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;

  // resident bookkeeping
  int n_uploaded = 0;
  std::vector<DevScene> res_host;    // host mirror of resident geometry
  std::vector<GraphEntry> graphs;
  std::string err;
};

namespace {

thread_local std::string g_init_err;   // failures of plan_init (no context yet)

int fail(plan_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_init_err = buf;
  return code;
}

#define CU(ctx, call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), PLAN_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                   \
  } while (0)

template <class T>
int dalloc(plan_ctx* ctx, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, PLAN_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  ctx->allocs.push_back(p);
  ctx->arena_bytes += count * sizeof(T);
  *ptr = static_cast<T*>(p);
  return PLAN_OK;
}

#define TRY(x)                    \
  do {                            \
    int s_ = (x);                 \
    if (s_ != PLAN_OK) return s_; \
  } while (0)

int alloc_set(plan_ctx* ctx, SceneSet& s, bool with_scenes) {
  const plan_config& c = ctx->cfg;
  if (with_scenes) {
    TRY(dalloc(ctx, &s.scenes, c.max_scenes));
    TRY(dalloc(ctx, &s.obs, size_t(c.max_scenes) * (c.max_obs > 0 ? c.max_obs : 1) * 6));
  }
  TRY(dalloc(ctx, &s.layout, c.max_scenes));
  TRY(dalloc(ctx, &s.tiles, size_t(c.max_samples) + c.max_scenes));
  TRY(dalloc(ctx, &s.sample_scene, c.max_samples));
  return PLAN_OK;
}

int validate_config(const plan_config* cfg, std::string* why) {
  char b[256];
  auto bad = [&](const char* m) { *why = m; return PLAN_EINVAL; };
  if (!cfg) return bad("cfg is NULL");
  if (const char* why_lower = lower_config_invalid(*cfg)) return bad(why_lower);
  if (cfg->outer_iters < 1 || cfg->outer_iters > 65535) return bad("outer_iters must be in [1, 65535]");
  if (cfg->n_elite < 1) return bad("n_elite must be >= 1");
  if (cfg->n_elite_c > kMaxEliteC || (cfg->n_elite_c <= 0 && 3 * cfg->n_elite > kMaxEliteC))
    return bad("n_elite_c must be <= 2048");
  if (cfg->n_elite_c > 0 && cfg->n_elite > cfg->n_elite_c) return bad("n_elite must be <= n_elite_c");
  if (cfg->prec < PLAN_PREC_FP64 || cfg->prec > PLAN_PREC_TF32X3) return bad("unknown prec");
  if (cfg->prec == PLAN_PREC_FP32 && !fused_supported(cfg->n_coef, cfg->m))
    return bad("the FP32 fused kernel supports n_coef in {8, 11, 16}");
  if (cfg->prec >= PLAN_PREC_TF32 && !tc_supported(cfg->n_coef, cfg->m, cfg->max_obs))
    return bad("the tensor-core modes support n_coef in {8, 11, 16} and m <= 128");
  if (cfg->max_obs < 0 || cfg->max_obs > kMaxObs) return bad("max_obs must be in [0, 64]");
  if (cfg->max_samples < 1 || cfg->max_samples > (1 << 24)) return bad("max_samples must be in [1, 2^24]");
  if (cfg->max_scenes < 1 || cfg->max_scenes > 65535) return bad("max_scenes must be in [1, 65535]");
  if (!(cfg->gamma > 0)) return bad("gamma must be > 0");
  if (!(cfg->eta > 0 && cfg->eta <= 1)) return bad("eta must be in (0, 1]");
  if (!(cfg->cov_eps >= 0)) return bad("cov_eps must be >= 0");
  if (!(cfg->v_des_hi >= cfg->v_des_lo) || !std::isfinite(cfg->v_des_lo) ||
      !std::isfinite(cfg->v_des_hi))
    return bad("v_des_hi must be >= v_des_lo (finite)");
  (void)b;
  return PLAN_OK;
}

int check_scene(plan_ctx* ctx, const plan_scene* s, int idx) {
  if (!s) return fail(ctx, PLAN_EINVAL, "scene %d is NULL", idx);
  if (s->n_obs > ctx->cfg.max_obs)
    return fail(ctx, PLAN_ECAPACITY, "scene %d: n_obs %d exceeds max_obs %d", idx, s->n_obs,
                ctx->cfg.max_obs);
  if (const char* why = scene_invalid(*s, ctx->cfg.lane_margin))
    return fail(ctx, PLAN_EINVAL, "scene %d: %s", idx, why);
  return PLAN_OK;
}

DevScene to_dev(const plan_ctx* ctx, const plan_scene& s, int obs_off) {
  DevScene d{};
  d.ego[0] = s.ego.x; d.ego[1] = s.ego.y; d.ego[2] = s.ego.vx;
  d.ego[3] = s.ego.vy; d.ego[4] = s.ego.ax; d.ego[5] = s.ego.ay;
  d.y_lb = ctx->cfg.lane_margin;
  d.y_ub = s.n_lanes * s.lane_width - ctx->cfg.lane_margin;
  d.kappa_road = s.kappa_road;
  d.lane_width = s.lane_width;
  d.n_lanes = s.n_lanes;
  d.n_obs = s.n_obs;
  d.obs_off = obs_off;
  fill_road(d, s, ctx->cfg.lane_margin);
  return d;
}

// Make the pinned staging buffer reusable (its previous copy has completed)
// and at least `bytes` large.
int stage_acquire(plan_ctx* ctx, size_t bytes) {
  if (ctx->stage_pending) {
    CU(ctx, cudaEventSynchronize(ctx->stage_done));
    ctx->stage_pending = false;
  }
  if (bytes > ctx->stage_bytes) {
    if (ctx->stage) cudaFreeHost(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, PLAN_ENOMEM, "pinned staging allocation of %zu bytes failed", bytes);
    }
    ctx->stage = static_cast<unsigned char*>(p);
    ctx->stage_bytes = bytes;
  }
  return PLAN_OK;
}

int stage_release(plan_ctx* ctx, cudaStream_t s) {
  CU(ctx, cudaEventRecord(ctx->stage_done, s));
  ctx->stage_pending = true;
  return PLAN_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Tiles of `warps` samples per CTA, never crossing a scene.
void make_tiles(const std::vector<int>& B, int warps, std::vector<Tile>* tiles,
                std::vector<Layout>* layout, std::vector<int>* sample_scene) {
  int off = 0;
  for (size_t s = 0; s < B.size(); ++s) {
    layout->push_back(Layout{B[s], off});
    for (int f = 0; f < B[s]; f += warps)
      tiles->push_back(Tile{int(s), f, std::min(warps, B[s] - f), 0});
    for (int j = 0; j < B[s]; ++j) sample_scene->push_back(int(s));
    off += B[s];
  }
}

struct Shape {
  int wps, spc;
};

// Fused-kernel shape: explicit tuning if set, else a heuristic that keeps
// about 16 warps per SM busy for small batches.
Shape pick_shape(const plan_ctx* ctx, int total_B) {
  if (ctx->cfg.prec >= PLAN_PREC_TF32) return Shape{1, tc_samples_per_cta()};
  if (ctx->tune_wps > 0 && ctx->tune_spc > 0) return Shape{ctx->tune_wps, ctx->tune_spc};
  // measured on the GB300: long horizons run best with two warps per sample,
  // two samples per CTA (one staged basis for both); otherwise one warp per
  // sample and, while the launch fits one CTA per SM, the fewest samples per
  // CTA that do (B = 1000 on 152 SMs: 7 per CTA, 143 CTAs, 1 % faster than
  // 125 CTAs of 8), else 4 per CTA
  if (ctx->cfg.m > 128) return Shape{2, 2};
  if (total_B <= 8 * ctx->sms) return Shape{1, std::max(1, (total_B + ctx->sms - 1) / ctx->sms)};
  return Shape{1, 4};
}

int pick_warps(const plan_ctx* ctx, int total_B) { return pick_shape(ctx, total_B).spc; }

// Upload scenes (geometry + obstacles) and the layout of B into `set`.  For the
// transient set (`tr`), an upload whose bytes equal the previous one's is
// skipped: the stream waits on the event recorded after those copies, so a
// repeated solve of the same scenes and sample counts enqueues no copies.
int upload(plan_ctx* ctx, SceneSet& set, const plan_scene* scenes, int S, const std::vector<int>* B,
           cudaStream_t s, std::vector<DevScene>* mirror) {
  std::vector<DevScene> ds;
  std::vector<double> ob;
  if (scenes) {
    set.road = false;
    for (int i = 0; i < S; ++i) {
      set.road = set.road || scenes[i].n_road > 0;
      ds.push_back(to_dev(ctx, scenes[i], int(ob.size() / 6)));
      for (int k = 0; k < scenes[i].n_obs; ++k) {
        const plan_obstacle& o = scenes[i].obs[k];
        ob.insert(ob.end(), {o.x0, o.y0, o.vx, o.vy, o.a, o.b});
      }
    }
  }
  std::vector<Tile> tiles;
  std::vector<Layout> layout;
  std::vector<int> ss;
  int total = 0;
  if (B) {
    for (int b : *B) total += b;
    make_tiles(*B, pick_warps(ctx, total), &tiles, &layout, &ss);
  }
  const size_t n1 = ds.size() * sizeof(DevScene), n2 = ob.size() * sizeof(double);
  const size_t n3 = layout.size() * sizeof(Layout), n4 = tiles.size() * sizeof(Tile);
  const size_t n5 = ss.size() * sizeof(int);
  const bool transient = &set == &ctx->tr;
  std::vector<unsigned char> key;
  if (transient) {
    const size_t counts[5] = {n1, n2, n3, n4, n5};
    key.reserve(n1 + n2 + n3 + n4 + n5 + sizeof counts);
    auto put = [&](const void* p, size_t n) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      key.insert(key.end(), b, b + n);
    };
    put(counts, sizeof counts);
    put(ds.data(), n1); put(ob.data(), n2); put(layout.data(), n3);
    put(tiles.data(), n4); put(ss.data(), n5);
    if (ctx->tr_key_ok && key == ctx->tr_key) {
      CU(ctx, cudaStreamWaitEvent(s, ctx->tr_ready, 0));
      if (mirror) *mirror = ds;
      return PLAN_OK;
    }
    ctx->tr_key_ok = false;     // set again once the new copies are enqueued
  }
  const size_t o2 = align_up(n1), o3 = o2 + align_up(n2), o4 = o3 + align_up(n3),
               o5 = o4 + align_up(n4), tot = o5 + align_up(n5);
  TRY(stage_acquire(ctx, tot));
  std::memcpy(ctx->stage, ds.data(), n1);
  std::memcpy(ctx->stage + o2, ob.data(), n2);
  std::memcpy(ctx->stage + o3, layout.data(), n3);
  std::memcpy(ctx->stage + o4, tiles.data(), n4);
  std::memcpy(ctx->stage + o5, ss.data(), n5);
  if (n1) CU(ctx, cudaMemcpyAsync(set.scenes, ctx->stage, n1, cudaMemcpyHostToDevice, s));
  if (n2) CU(ctx, cudaMemcpyAsync(set.obs, ctx->stage + o2, n2, cudaMemcpyHostToDevice, s));
  if (n3) CU(ctx, cudaMemcpyAsync(set.layout, ctx->stage + o3, n3, cudaMemcpyHostToDevice, s));
  if (n4) CU(ctx, cudaMemcpyAsync(set.tiles, ctx->stage + o4, n4, cudaMemcpyHostToDevice, s));
  if (n5) CU(ctx, cudaMemcpyAsync(set.sample_scene, ctx->stage + o5, n5, cudaMemcpyHostToDevice, s));
  TRY(stage_release(ctx, s));
  if (transient) {
    CU(ctx, cudaEventRecord(ctx->tr_ready, s));
    ctx->tr_key = std::move(key);
    ctx->tr_key_ok = true;
  }
  if (mirror) *mirror = ds;
  return PLAN_OK;
}

// Lower-level solve of all samples described by `set` (Alg. 1 lines 6-9).
// status: per-sample PLAN_OK / PLAN_ENONFINITE, or NULL.
cudaError_t run_solve(plan_ctx* ctx, const SceneSet& set, const SceneSet& lay, int n_tiles,
                      int total_B, int n_scenes, const double* p, double* xi, double* r, double* cu,
                      int* status, cudaStream_t s) {
  if (ctx->cfg.prec == PLAN_PREC_FP32) {
    const Shape sh = pick_shape(ctx, total_B);
    FusedLaunch L{};
    L.scenes = set.scenes;
    L.layout = lay.layout;
    L.obs = set.obs;
    L.tiles = lay.tiles;
    L.n_tiles = n_tiles;
    L.sample_scene = lay.sample_scene;
    L.total = total_B;
    L.work = ctx->work;
    L.sms = ctx->sms;
    // automatic choice: the persistent form only for one scene; in the
    // graph-captured cycle of a 256-scene batch it measured 1-2 % slower than
    // one tile per CTA, so scene mixes keep the tiles
    L.persist = ctx->persist == PLAN_PERSIST_AUTO && n_scenes > 1 ? PLAN_PERSIST_OFF : ctx->persist;
    L.wps = sh.wps;
    L.spc = sh.spc;
    L.road = set.road;
    L.p = p;
    L.xi = xi;
    L.r = r;
    L.cu = cu;
    L.st = status;
    return launch_fused_f32(L, ctx->c, ctx->prm, s);
  }
  if (ctx->cfg.prec >= PLAN_PREC_TF32)
    return launch_tc(ctx->cfg.prec, set.scenes, lay.layout, set.obs, lay.tiles, n_tiles, p, ctx->c,
                     ctx->prm, xi, r, cu, status, ctx->tc_err, s);
  return launch_plain64(set.scenes, lay.layout, lay.sample_scene, set.obs, total_B, p, ctx->c,
                        ctx->prm, ctx->pw, xi, r, cu, status, s);
}

int n_tiles_of(const std::vector<int>& B, int warps) {
  int n = 0;
  for (int b : B) n += (b + warps - 1) / warps;
  return n;
}

void chol_host(const double* A, double eps, int d, double* L, bool* ok) {
  *ok = true;
  for (int i = 0; i < kMaxDp * kMaxDp; ++i) L[i] = 0.0;
  for (int j = 0; j < d; ++j) {
    double s = A[j * kMaxDp + j] + eps;
    for (int k = 0; k < j; ++k) s -= L[j * kMaxDp + k] * L[j * kMaxDp + k];
    if (!(s > 0)) { *ok = false; return; }
    const double dj = std::sqrt(s);
    L[j * kMaxDp + j] = dj;
    for (int i = j + 1; i < d; ++i) {
      double v = A[i * kMaxDp + j];
      for (int k = 0; k < j; ++k) v -= L[i * kMaxDp + k] * L[j * kMaxDp + k];
      L[i * kMaxDp + j] = v / dj;
    }
  }
}

// DevCem from a host state; the initial moments of a fresh episode follow
// from the uniform first-iteration distribution of the scene's lanes (and,
// with goal entries, of x_f = ego_x + U[v_des_lo, v_des_hi] t_f and a
// lane-centre y_f).
int make_cem(plan_ctx* ctx, const plan_cem_state* st, int n_lanes, double lane_width, double ego_x,
             DevCem* out) {
  const int ns = ctx->cfg.n_seg, d = ctx->prm.d_p;
  DevCem c{};
  c.seed = st->seed;
  c.step = st->episode_step;
  c.fresh = st->fresh ? 1 : 0;
  if (c.fresh) {
    const double L = n_lanes, w = lane_width;
    const double lo = ctx->cfg.v_des_lo, hi = ctx->cfg.v_des_hi;
    const double lane_mu = L * w / 2.0, lane_var = w * w * (L * L - 1.0) / 12.0;
    const double v_mu = 0.5 * (lo + hi), v_var = (hi - lo) * (hi - lo) / 12.0;
    for (int e = 0; e < ns; ++e) {
      c.mu[e] = lane_mu;
      c.mu[ns + e] = v_mu;
      c.sigma[e * kMaxDp + e] = lane_var;
      c.sigma[(ns + e) * kMaxDp + ns + e] = v_var;
    }
    if (ctx->cfg.goal) {
      const double tf = (ctx->cfg.m - 1) * ctx->cfg.dt;
      c.mu[2 * ns] = ego_x + tf * v_mu;
      c.sigma[(2 * ns) * kMaxDp + 2 * ns] = tf * tf * v_var;
      c.mu[2 * ns + 1] = lane_mu;
      c.sigma[(2 * ns + 1) * kMaxDp + 2 * ns + 1] = lane_var;
    }
  } else {
    for (int a = 0; a < d; ++a) {
      c.mu[a] = st->mu[a];
      for (int b = 0; b < d; ++b) c.sigma[a * kMaxDp + b] = st->sigma[a * PLAN_MAX_DP + b];
    }
  }
  for (int a = 0; a < d; ++a)
    if (!std::isfinite(c.mu[a])) return fail(ctx, PLAN_EINVAL, "mu not finite");
  bool ok = true;
  chol_host(c.sigma, ctx->cfg.cov_eps, d, c.chol, &ok);
  if (!ok && !c.fresh) return fail(ctx, PLAN_EINVAL, "sigma + cov_eps I is not positive definite");
  *out = c;
  return PLAN_OK;
}

}  // namespace

void plan::set_unbound_error(const char* msg) { g_init_err = msg; }

// ----------------------------------------------------------------- serving hooks

size_t plan::ctx_bytes(const plan_ctx* ctx) { return ctx->arena_bytes; }

const char* plan::ctx_error(const plan_ctx* ctx) { return ctx->err.c_str(); }

int plan::ctx_make_state(plan_ctx* ctx, const plan_cem_state* st, int n_lanes, double lane_width,
                         double ego_x, DevCem* out) {
  return make_cem(ctx, st, n_lanes, lane_width, ego_x, out);
}

int plan::ctx_wave(plan_ctx* ctx, const plan_scene* scenes, const int* B, int S,
                   const DevCem* init, const int* gather, const int* scatter, DevCem* table,
                   DevCem* results, cudaStream_t s) {
  if (S < 1 || S > ctx->cfg.max_scenes) return fail(ctx, PLAN_ECAPACITY, "wave of %d scenes", S);
  std::vector<int> Bv(B, B + S);
  long long total = 0;
  int max_B = 0;
  for (int i = 0; i < S; ++i) {
    if (Bv[i] < 1) return fail(ctx, PLAN_EINVAL, "B[%d] must be >= 1", i);
    total += Bv[i];
    max_B = std::max(max_B, Bv[i]);
    TRY(check_scene(ctx, &scenes[i], i));
  }
  if (total > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "wave exceeds max_samples");
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(upload(ctx, ctx->res, scenes, S, &Bv, s, &ctx->res_host));
  ctx->n_uploaded = S;
  const size_t nb = sizeof(DevCem) * S, ni = sizeof(int) * S;
  TRY(stage_acquire(ctx, nb + 2 * ni));
  std::memcpy(ctx->stage, init, nb);
  std::memcpy(ctx->stage + nb, gather, ni);
  std::memcpy(ctx->stage + nb + ni, scatter, ni);
  CU(ctx, cudaMemcpyAsync(ctx->cem, ctx->stage, nb, cudaMemcpyHostToDevice, s));
  CU(ctx, cudaMemcpyAsync(ctx->rows, ctx->stage + nb, 2 * ni, cudaMemcpyHostToDevice, s));
  TRY(stage_release(ctx, s));
  CU(ctx, launch_cem_copy(ctx->cem, table, ctx->rows, S, false, s));
  const int nt = n_tiles_of(Bv, pick_warps(ctx, int(total)));
  for (int l = 1; l <= ctx->cfg.outer_iters; ++l) {
    CU(ctx, launch_sample(ctx->res.scenes, ctx->res.layout, ctx->cem, S, max_B, l, ctx->prm, ctx->p, s));
    CU(ctx, run_solve(ctx, ctx->res, ctx->res, nt, int(total), S, ctx->p, ctx->xi, ctx->r,
                      ctx->cu, nullptr, s));
    CU(ctx, launch_select_update(ctx->res.layout, ctx->cem, S, l, ctx->prm, ctx->p, ctx->xi,
                                 ctx->r, ctx->cu, ctx->elite, max_B, s));
  }
  CU(ctx, launch_cem_copy(table, ctx->cem, ctx->rows + S, S, true, s));
  CU(ctx, cudaMemcpyAsync(results, ctx->cem, nb, cudaMemcpyDeviceToHost, s));
  return PLAN_OK;
}

extern "C" {

const char* plan_status_str(int status) {
  switch (status) {
    case PLAN_OK: return "ok";
    case PLAN_EINVAL: return "invalid argument";
    case PLAN_ENOMEM: return "out of memory";
    case PLAN_ECAPACITY: return "capacity exceeded";
    case PLAN_ETIMEOUT: return "timed out";
    case PLAN_ECUDA: return "CUDA error";
    case PLAN_ESTATE: return "invalid state";
    case PLAN_ENONFINITE: return "non-finite result";
    default: return "unknown status";
  }
}

int plan_last_error(const plan_ctx* ctx, char* buf, size_t len) {
  if (!buf || len == 0) return PLAN_EINVAL;
  std::snprintf(buf, len, "%s", ctx ? ctx->err.c_str() : g_init_err.c_str());
  return PLAN_OK;
}

int plan_destroy(plan_ctx* ctx) {
  if (!ctx) return PLAN_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(ctx->device);
  if (ctx->internal) cudaStreamSynchronize(ctx->internal);
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  if (ctx->io) cudaFreeHost(ctx->io);
  if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
  if (ctx->tr_ready) cudaEventDestroy(ctx->tr_ready);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->internal) cudaStreamDestroy(ctx->internal);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  cudaSetDevice(dev);
  delete ctx;
  return PLAN_OK;
}

int plan_init(const plan_config* cfg, plan_ctx** out) {
  if (!out) return PLAN_EINVAL;
  *out = nullptr;
  std::string why;
  if (validate_config(cfg, &why) != PLAN_OK) return fail(nullptr, PLAN_EINVAL, "%s", why.c_str());
  plan_ctx* ctx = new (std::nothrow) plan_ctx();
  if (!ctx) return PLAN_ENOMEM;
  ctx->cfg = *cfg;
  const plan_config& c = *cfg;
  Params& p = ctx->prm;
  p.m = c.m; p.n = c.n_coef; p.n_seg = c.n_seg; p.K = c.inner_iters; p.L = c.outer_iters;
  p.q = c.n_elite; p.n_c = c.n_elite_c > 0 ? c.n_elite_c : 3 * c.n_elite;
  p.d_p = 2 * c.n_seg + 2 * c.goal; p.max_obs = c.max_obs; p.goal = c.goal;
  p.dt = c.dt; p.rho = c.rho; p.kp_lat = c.kp_lat; p.kv_lat = c.kv_lat; p.kp_lon = c.kp_lon;
  p.gamma = c.gamma; p.eta = c.eta; p.cov_eps = c.cov_eps; p.v_min = c.v_min; p.v_max = c.v_max;
  p.a_max = c.a_max; p.kappa_max = c.kappa_max; p.c_max = c.c_max; p.lane_margin = c.lane_margin;
  p.v_des_lo = c.v_des_lo; p.v_des_hi = c.v_des_hi;

  auto bail = [&](int code) {
    g_init_err = ctx->err.empty() ? "CUDA initialisation failed" : ctx->err;
    plan_destroy(ctx);
    return code;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(PLAN_ECUDA);
  }
  if (cudaStreamCreateWithFlags(&ctx->internal, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->tr_ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(PLAN_ECUDA);
  }
  const int m = c.m, n = c.n_coef, ns = c.n_seg, d = p.d_p;
  const size_t B = c.max_samples;
  Consts& k = ctx->c;
  k.m = m; k.n = n; k.n_seg = ns; k.max_obs = c.max_obs;
  k.goal = c.goal; k.ne = 3 + 2 * c.goal;
  int st = PLAN_OK;
  auto A = [&](int s) { if (st == PLAN_OK) st = s; };
  A(dalloc(ctx, &k.basis64, size_t(3) * m * n));
  A(dalloc(ctx, &k.basis32, size_t(m) * basis32_stride(n)));
  A(dalloc(ctx, &k.s1_64, size_t(2) * n * (ns + k.ne)));
  A(dalloc(ctx, &k.s1_32, size_t(2) * n * (ns + k.ne)));
  A(dalloc(ctx, &k.pj64, size_t(c.max_obs + 1) * 2 * n * (2 * n + k.ne)));
  A(dalloc(ctx, &k.pj32, size_t(c.max_obs + 1) * 2 * n * (2 * n + k.ne)));
  if (st == PLAN_OK) A(alloc_set(ctx, ctx->tr, true));
  if (st == PLAN_OK) A(alloc_set(ctx, ctx->res, true));
  A(dalloc(ctx, &ctx->cem, c.max_scenes));
  A(dalloc(ctx, &ctx->cem_tmp, 1));
  A(dalloc(ctx, &ctx->layout_tmp, 1));
  A(dalloc(ctx, &ctx->p, B * d));
  A(dalloc(ctx, &ctx->xi, B * 2 * n));
  A(dalloc(ctx, &ctx->r, B));
  A(dalloc(ctx, &ctx->cu, B));
  A(dalloc(ctx, &ctx->elite, size_t(c.max_scenes) * c.n_elite));
  A(dalloc(ctx, &ctx->rows, size_t(2) * c.max_scenes));
  A(dalloc(ctx, &ctx->tc_err, 1));
  A(dalloc(ctx, &ctx->work, 2));
  if (c.outer_iters > 1) A(dalloc(ctx, &ctx->zbuf, B * d));
  if (c.prec == PLAN_PREC_FP64) {
    A(dalloc(ctx, &ctx->pw.xibarp, B * 32));
    A(dalloc(ctx, &ctx->pw.xi, B * 32));
    A(dalloc(ctx, &ctx->pw.lam, B * 32));
    A(dalloc(ctx, &ctx->pw.w, B * 32));
    A(dalloc(ctx, &ctx->pw.state, B * 6 * m));
    A(dalloc(ctx, &ctx->pw.eps, B * 7 * m));
    A(dalloc(ctx, &ctx->pw.da, B * m));
    A(dalloc(ctx, &ctx->pw.xprev, B * m));
  }
  if (st != PLAN_OK) return bail(st);
  {
    ctx->io_obs = align_up(sizeof(DevScene));
    ctx->io_cem = ctx->io_obs + align_up(size_t(c.max_obs) * 6 * sizeof(double));
    ctx->io_ret = ctx->io_cem + align_up(sizeof(DevCem));
    const size_t io_bytes = ctx->io_ret + align_up(sizeof(DevCem) + sizeof(unsigned long long));
    void* h = nullptr;
    if (cudaHostAlloc(&h, io_bytes, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return bail(PLAN_ENOMEM);
    }
    ctx->io = static_cast<unsigned char*>(h);
    std::memset(ctx->io, 0, io_bytes);
    if (cudaHostGetDevicePointer(&ctx->io_dev, h, 0) != cudaSuccess) {
      cudaGetLastError();
      return bail(PLAN_ECUDA);
    }
  }
  cem_setup();
  fused_setup();
  if (c.prec >= PLAN_PREC_TF32) tc_setup();
  if (build_constants(k, p, ctx->internal) != cudaSuccess ||
      cudaMemsetAsync(ctx->cem, 0, sizeof(DevCem) * c.max_scenes, ctx->internal) != cudaSuccess ||
      cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->internal) != cudaSuccess ||
      cudaMemsetAsync(ctx->work, 0, 2 * sizeof(int), ctx->internal) != cudaSuccess ||
      cudaStreamSynchronize(ctx->internal) != cudaSuccess) {
    cudaGetLastError();
    return bail(PLAN_ECUDA);
  }
  *out = ctx;
  return PLAN_OK;
}

int plan_solve_batch(plan_ctx* ctx, const plan_scene* scenes, const int* B, int S, const double* p,
                     double* xi, double* resid, double* cu, int* status, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (S < 0 || (S > 0 && (!scenes || !B))) return fail(ctx, PLAN_EINVAL, "bad scenes / B");
  if (S > ctx->cfg.max_scenes) return fail(ctx, PLAN_ECAPACITY, "S exceeds max_scenes");
  std::vector<int> Bv(B, B + S);
  long long total = 0;
  for (int i = 0; i < S; ++i) {
    if (Bv[i] < 0) return fail(ctx, PLAN_EINVAL, "B[%d] < 0", i);
    total += Bv[i];
    TRY(check_scene(ctx, &scenes[i], i));
  }
  if (total > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "samples exceed max_samples");
  if (total == 0) return PLAN_OK;
  if (!p || !resid || !cu) return fail(ctx, PLAN_EINVAL, "p, resid and cu must be non-NULL");
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(upload(ctx, ctx->tr, scenes, S, &Bv, s, nullptr));
  const int spc = pick_warps(ctx, int(total));
  CU(ctx, run_solve(ctx, ctx->tr, ctx->tr, n_tiles_of(Bv, spc), int(total), S, p, xi, resid,
                    cu, status, s));
  return PLAN_OK;
}

int plan_solve(plan_ctx* ctx, const plan_scene* scene, const double* p, int B, double* xi,
               double* resid, double* cu, int* status, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  return plan_solve_batch(ctx, scene, &B, 1, p, xi, resid, cu, status, stream);
}

int plan_upload_scenes(plan_ctx* ctx, const plan_scene* scenes, int S, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (S < 1 || !scenes) return fail(ctx, PLAN_EINVAL, "need S >= 1 scenes");
  if (S > ctx->cfg.max_scenes) return fail(ctx, PLAN_ECAPACITY, "S exceeds max_scenes");
  for (int i = 0; i < S; ++i) TRY(check_scene(ctx, &scenes[i], i));
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(upload(ctx, ctx->res, scenes, S, nullptr, static_cast<cudaStream_t>(stream), &ctx->res_host));
  ctx->n_uploaded = S;
  return PLAN_OK;
}

int plan_set_state(plan_ctx* ctx, int slot, const plan_cem_state* st, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!st) return fail(ctx, PLAN_EINVAL, "state is NULL");
  if (slot < 0 || slot >= ctx->n_uploaded)
    return fail(ctx, PLAN_ESTATE, "slot %d has no uploaded scene", slot);
  DevCem c;
  TRY(make_cem(ctx, st, ctx->res_host[slot].n_lanes, ctx->res_host[slot].lane_width,
               ctx->res_host[slot].ego[0], &c));
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(stage_acquire(ctx, sizeof(DevCem)));
  std::memcpy(ctx->stage, &c, sizeof c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU(ctx, cudaMemcpyAsync(ctx->cem + slot, ctx->stage, sizeof c, cudaMemcpyHostToDevice, s));
  // the factor of an imported covariance is taken again on the device, by the
  // routine that factored it in the interrupted episode (reciprocal square
  // roots; the host's, with square root and division, differs in the last bits)
  CU(ctx, launch_import_chol(ctx->cem + slot, ctx->prm, s));
  return stage_release(ctx, s);
}

void cem_to_state(const plan_ctx* ctx, const DevCem& c, plan_cem_state* st) {
  const int d = ctx->prm.d_p;
  std::memset(st, 0, sizeof *st);
  for (int a = 0; a < d; ++a) {
    st->mu[a] = c.mu[a];
    for (int b = 0; b < d; ++b) st->sigma[a * PLAN_MAX_DP + b] = c.sigma[a * kMaxDp + b];
  }
  st->seed = c.seed;
  st->episode_step = c.step;
  st->fresh = c.fresh;
}

void cem_to_result(const plan_ctx* ctx, const DevCem& c, plan_result* out) {
  std::memset(out, 0, sizeof *out);
  for (int a = 0; a < ctx->prm.d_p; ++a) out->p[a] = c.best_p[a];
  for (int a = 0; a < 2 * ctx->cfg.n_coef; ++a) out->xi[a] = c.best_xi[a];
  out->cost = c.best_cost;
  out->resid = c.best_r;
  out->cu = c.best_cu;
  out->index = c.best_index;
}

int plan_get_state(plan_ctx* ctx, int slot, plan_cem_state* st, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!st || slot < 0 || slot >= ctx->cfg.max_scenes) return fail(ctx, PLAN_EINVAL, "bad slot/state");
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(stage_acquire(ctx, sizeof(DevCem) + sizeof(int)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU(ctx, cudaMemcpyAsync(ctx->stage, ctx->cem + slot, sizeof(DevCem), cudaMemcpyDeviceToHost, s));
  CU(ctx, cudaMemcpyAsync(ctx->stage + sizeof(DevCem), ctx->tc_err, sizeof(int),
                          cudaMemcpyDeviceToHost, s));
  CU(ctx, cudaStreamSynchronize(s));
  DevCem c;
  std::memcpy(&c, ctx->stage, sizeof c);
  int tc_timeout = 0;
  std::memcpy(&tc_timeout, ctx->stage + sizeof c, sizeof tc_timeout);
  if (tc_timeout) {
    // report once: clear the flag for the next calls
    cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s);
    return fail(ctx, PLAN_ETIMEOUT, "a tensor-core wait of the solve timed out");
  }
  cem_to_state(ctx, c, st);
  return PLAN_OK;
}

int plan_get_result(plan_ctx* ctx, int slot, plan_result* out, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!out || slot < 0 || slot >= ctx->cfg.max_scenes) return fail(ctx, PLAN_EINVAL, "bad slot/out");
  CU(ctx, cudaSetDevice(ctx->device));
  TRY(stage_acquire(ctx, sizeof(DevCem) + sizeof(int)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU(ctx, cudaMemcpyAsync(ctx->stage, ctx->cem + slot, sizeof(DevCem), cudaMemcpyDeviceToHost, s));
  CU(ctx, cudaMemcpyAsync(ctx->stage + sizeof(DevCem), ctx->tc_err, sizeof(int),
                          cudaMemcpyDeviceToHost, s));
  CU(ctx, cudaStreamSynchronize(s));
  DevCem c;
  std::memcpy(&c, ctx->stage, sizeof c);
  int tc_timeout = 0;
  std::memcpy(&tc_timeout, ctx->stage + sizeof c, sizeof tc_timeout);
  if (tc_timeout) {
    // report once: clear the flag for the next calls
    cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s);
    return fail(ctx, PLAN_ETIMEOUT, "a tensor-core wait of the solve timed out");
  }
  cem_to_result(ctx, c, out);
  if (!std::isfinite(c.best_cost)) return fail(ctx, PLAN_ENONFINITE, "best cost is not finite");
  return PLAN_OK;
}

namespace {

// Alg. 1 on the resident scene slots 0..S-1 as one captured graph per sample
// layout; io: the graph also moves plan_step's staging in at its head and out
// at its tail (through the host-mapped buffer), so that cycle needs no copies.
int run_cycle(plan_ctx* ctx, const int* B, int S, void* stream, bool io) {
  if (S < 1 || !B) return fail(ctx, PLAN_EINVAL, "need S >= 1 and B");
  if (S > ctx->n_uploaded) return fail(ctx, PLAN_ECAPACITY, "S exceeds the uploaded scene slots");
  std::vector<int> Bv(B, B + S);
  long long total = 0;
  int max_B = 0;
  for (int i = 0; i < S; ++i) {
    if (Bv[i] < 1) return fail(ctx, PLAN_EINVAL, "B[%d] must be >= 1", i);
    total += Bv[i];
    max_B = std::max(max_B, Bv[i]);
  }
  if (total > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "samples exceed max_samples");
  CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GraphEntry* g = nullptr;
  for (auto& e : ctx->graphs)
    if (e.B == Bv && e.road == ctx->res.road && e.io == io) g = &e;
  if (!g) {
    GraphEntry e;
    e.B = Bv;
    e.road = ctx->res.road;
    e.io = io;
    e.total_B = int(total);
    e.max_B = max_B;
    e.set.scenes = ctx->res.scenes;
    e.set.obs = ctx->res.obs;
    e.set.road = ctx->res.road;
    TRY(dalloc(ctx, &e.set.layout, S));
    TRY(dalloc(ctx, &e.set.tiles, size_t(total) + S));
    TRY(dalloc(ctx, &e.set.sample_scene, size_t(total)));
    TRY(upload(ctx, e.set, nullptr, 0, &Bv, ctx->internal, nullptr));
    CU(ctx, cudaStreamSynchronize(ctx->internal));
    const int nt = n_tiles_of(Bv, pick_warps(ctx, int(total)));
    cudaGraph_t graph = nullptr;
    CU(ctx, cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    if (io)
      ce = launch_io_in(ctx->io_dev, ctx->io_obs, ctx->io_cem, e.set.scenes, e.set.obs, ctx->cem,
                        ctx->prm, ctx->capture);
    const int L = ctx->cfg.outer_iters;
    for (int l = 1; l <= L && ce == cudaSuccess; ++l) {
      // the normals of iteration l >= 2 were drawn on the side stream beside
      // the previous solve: join that branch before sampling
      if (l >= 2) ce = cudaStreamWaitEvent(ctx->capture, ctx->join_ev, 0);
      // after the staging kernel the first sampling waits for it in full (its
      // writes are read by the solve's prologue before that kernel's own wait)
      if (ce == cudaSuccess)
        ce = launch_sample(e.set.scenes, e.set.layout, ctx->cem, S, max_B, l, ctx->prm, ctx->p,
                           ctx->capture, !(io && l == 1), l >= 2 ? ctx->zbuf : nullptr);
      if (ce == cudaSuccess && l < L) {
        // fork: the normals of iteration l + 1 (they depend only on the seed
        // and the episode step) on the side stream, once this sampling has
        // read the buffer; the float64 draws then overlap the float32 solve
        ce = cudaEventRecord(ctx->fork_ev, ctx->capture);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0);
        if (ce == cudaSuccess)
          ce = launch_normals(e.set.layout, ctx->cem, S, max_B, l + 1, ctx->prm, ctx->zbuf,
                              ctx->side);
        if (ce == cudaSuccess) ce = cudaEventRecord(ctx->join_ev, ctx->side);
      }
      if (ce == cudaSuccess)
        ce = run_solve(ctx, e.set, e.set, nt, int(total), S, ctx->p, ctx->xi, ctx->r, ctx->cu,
                       nullptr, ctx->capture);
      if (ce == cudaSuccess)
        ce = launch_select_update(e.set.layout, ctx->cem, S, l, ctx->prm, ctx->p, ctx->xi, ctx->r,
                                  ctx->cu, ctx->elite, max_B, ctx->capture);
    }
    if (io && ce == cudaSuccess)
      ce = launch_io_out(ctx->cem, ctx->tc_err, ctx->io_dev, ctx->io_ret, ctx->capture);
    cudaError_t ee = cudaStreamEndCapture(ctx->capture, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(ctx, PLAN_ECUDA, "graph capture failed: %s",
                  cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, PLAN_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    }
    e.exec = exec;
    ctx->graphs.push_back(e);
    g = &ctx->graphs.back();
  }
  CU(ctx, cudaGraphLaunch(g->exec, s));
  return PLAN_OK;
}

}  // namespace

int plan_step_resident(plan_ctx* ctx, const int* B, int S, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  return run_cycle(ctx, B, S, stream, false);
}

int plan_step(plan_ctx* ctx, const plan_scene* scene, plan_cem_state* st, int B, plan_result* out,
              void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!scene || !st || !out) return fail(ctx, PLAN_EINVAL, "scene, state and out must be non-NULL");
  TRY(check_scene(ctx, scene, 0));
  if (B < 1 || B > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "B out of range");
  DevCem c0;
  TRY(make_cem(ctx, st, scene->n_lanes, scene->lane_width, scene->ego.x, &c0));
  CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scene, obstacles and state go into the host-mapped staging buffer; the
  // cycle's graph moves them in, runs Alg. 1 and moves the final state (with
  // the best pair) and the timeout flag back: one launch, one sync.  The
  // previous call synchronised, so no graph is still reading the buffer.
  const DevScene ds = to_dev(ctx, *scene, 0);
  std::memcpy(ctx->io, &ds, sizeof ds);
  double* ob = reinterpret_cast<double*>(ctx->io + ctx->io_obs);
  for (int k = 0; k < scene->n_obs; ++k) {
    const plan_obstacle& o = scene->obs[k];
    const double v[6] = {o.x0, o.y0, o.vx, o.vy, o.a, o.b};
    std::memcpy(ob + 6 * k, v, sizeof v);
  }
  std::memcpy(ctx->io + ctx->io_cem, &c0, sizeof c0);
  ctx->res.road = scene->n_road > 0;
  ctx->res_host.assign(1, ds);
  ctx->n_uploaded = 1;
  TRY(run_cycle(ctx, &B, 1, stream, true));
  CU(ctx, cudaStreamSynchronize(s));
  DevCem c;
  std::memcpy(&c, ctx->io + ctx->io_ret, sizeof c);
  unsigned long long tc_timeout = 0;
  std::memcpy(&tc_timeout, ctx->io + ctx->io_ret + sizeof c, sizeof tc_timeout);
  if (tc_timeout) {
    // report once: clear the flag for the next calls
    cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s);
    return fail(ctx, PLAN_ETIMEOUT, "a tensor-core wait of the solve timed out");
  }
  cem_to_result(ctx, c, out);
  cem_to_state(ctx, c, st);
  if (!std::isfinite(c.best_cost)) return fail(ctx, PLAN_ENONFINITE, "best cost is not finite");
  return PLAN_OK;
}

int plan_select_elites(plan_ctx* ctx, const double* resid, const double* cu, int B, int n_c, int q,
                       int* elite, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!resid || !cu || !elite) return fail(ctx, PLAN_EINVAL, "NULL buffer");
  if (B < 1 || n_c < 1 || n_c > B || n_c > kMaxEliteC || q < 1 || q > n_c)
    return fail(ctx, PLAN_EINVAL, "need 1 <= q <= n_c <= min(B, 2048)");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, launch_select_only(resid, cu, B, n_c, q, elite, static_cast<cudaStream_t>(stream)));
  return PLAN_OK;
}

int plan_update_distribution(plan_ctx* ctx, const double* p_elite, const double* cost, int q,
                             double* mu, double* sigma, void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!p_elite || !cost || !mu || !sigma) return fail(ctx, PLAN_EINVAL, "NULL buffer");
  if (q < 1 || q > kMaxEliteC) return fail(ctx, PLAN_EINVAL, "q must be in [1, 2048]");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, launch_update_only(p_elite, cost, q, ctx->prm.d_p, ctx->cfg.gamma, ctx->cfg.eta, mu,
                             sigma, static_cast<cudaStream_t>(stream)));
  return PLAN_OK;
}

int plan_probe_alu(double* out, void* stream) {
  if (!out) {
    set_unbound_error("out is NULL");
    return PLAN_EINVAL;
  }
  if (probe_alu(out, static_cast<cudaStream_t>(stream)) != 0) {
    set_unbound_error("probe launch failed");
    cudaGetLastError();
    return PLAN_ECUDA;
  }
  return PLAN_OK;
}

int plan_probe_tc_wide(int passes, int iters, double* out, void* stream) {
  if (!out) {
    set_unbound_error("NULL out");
    return PLAN_EINVAL;
  }
  if ((passes != 1 && passes != 3) || iters < 1 || iters > 10000) {
    set_unbound_error("passes must be 1 or 3 and iters in [1, 10000]");
    return PLAN_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    set_unbound_error("no CUDA device");
    return PLAN_ECUDA;
  }
  std::vector<double> cyc(size_t(5) * sms);
  int timed_out = 0;
  const cudaError_t e = tc_wide_probe(passes, iters, sms, cyc.data(),
                                      static_cast<cudaStream_t>(stream), &timed_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_unbound_error(cudaGetErrorString(e));
    return PLAN_ECUDA;
  }
  if (timed_out) {
    set_unbound_error("a bounded tensor-core wait gave up");
    return PLAN_ETIMEOUT;
  }
  for (int q = 0; q < 5; ++q) {
    std::vector<double> v(sms);
    for (int c = 0; c < sms; ++c) v[c] = cyc[size_t(5) * c + q];
    std::nth_element(v.begin(), v.begin() + sms / 2, v.end());
    out[q] = v[sms / 2];
  }
  out[5] = double(sms);
  return PLAN_OK;
}

int plan_probe_wait_timeout(int wait_us, void* stream) {
  if (wait_us < 1 || wait_us > 100000) {
    set_unbound_error("wait_us must be in [1, 100000]");
    return PLAN_EINVAL;
  }
  int timed_out = 0;
  // SM clock cycles: 2.1 per nanosecond bounds the wait from above at the maximum clock
  const cudaError_t e = wait_probe(2100LL * wait_us, static_cast<cudaStream_t>(stream), &timed_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_unbound_error(cudaGetErrorString(e));
    return PLAN_ECUDA;
  }
  if (timed_out) {
    set_unbound_error("the bounded wait gave up: no arrival on the mbarrier");
    return PLAN_ETIMEOUT;
  }
  return PLAN_OK;
}

int plan_qp_forward(plan_ctx* ctx, const double* p, const double* b0, int B, double* xi,
                    void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (B < 0) return fail(ctx, PLAN_EINVAL, "B must be >= 0");
  if (B > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "B exceeds max_samples");
  if (B == 0) return PLAN_OK;
  if (!p || !b0 || !xi) return fail(ctx, PLAN_EINVAL, "NULL buffer");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, launch_qp_forward(ctx->c, p, b0, B, xi, static_cast<cudaStream_t>(stream)));
  return PLAN_OK;
}

int plan_qp_backward(plan_ctx* ctx, const double* g, int B, double* grad_p, double* grad_b0,
                     void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (B < 0) return fail(ctx, PLAN_EINVAL, "B must be >= 0");
  if (B > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "B exceeds max_samples");
  if (B == 0) return PLAN_OK;
  if (!g || !grad_p) return fail(ctx, PLAN_EINVAL, "NULL buffer");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, launch_qp_backward(ctx->c, g, B, grad_p, grad_b0, static_cast<cudaStream_t>(stream)));
  return PLAN_OK;
}

int plan_sample(plan_ctx* ctx, const plan_scene* scene, const double* mu, const double* sigma,
                int fresh, int l, uint64_t seed, uint64_t episode_step, int B, double* p,
                void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!scene || !p || (!fresh && (!mu || !sigma))) return fail(ctx, PLAN_EINVAL, "NULL argument");
  if (l < 1 || l > 65535 || B < 0) return fail(ctx, PLAN_EINVAL, "bad l or B");
  if (B > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "B exceeds max_samples");
  TRY(check_scene(ctx, scene, 0));
  if (B == 0) return PLAN_OK;
  plan_cem_state st{};
  const int d = ctx->prm.d_p;
  if (!fresh)
    for (int a = 0; a < d; ++a) {
      st.mu[a] = mu[a];
      for (int b = 0; b < d; ++b) st.sigma[a * PLAN_MAX_DP + b] = sigma[a * d + b];
    }
  st.seed = seed;
  st.episode_step = episode_step;
  st.fresh = fresh;
  DevCem c;
  TRY(make_cem(ctx, &st, scene->n_lanes, scene->lane_width, scene->ego.x, &c));
  CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int> Bv{B};
  TRY(upload(ctx, ctx->tr, scene, 1, &Bv, s, nullptr));
  TRY(stage_acquire(ctx, sizeof(DevCem)));
  std::memcpy(ctx->stage, &c, sizeof c);
  CU(ctx, cudaMemcpyAsync(ctx->cem_tmp, ctx->stage, sizeof c, cudaMemcpyHostToDevice, s));
  TRY(stage_release(ctx, s));
  CU(ctx, launch_sample(ctx->tr.scenes, ctx->tr.layout, ctx->cem_tmp, 1, B, l, ctx->prm, p, s));
  return PLAN_OK;
}

int plan_set_tuning(plan_ctx* ctx, int warps_per_sample, int samples_per_cta) {
  if (!ctx) return PLAN_EINVAL;
  const bool automatic = warps_per_sample == 0 && samples_per_cta == 0;
  if (!automatic && !fused_shape_ok(warps_per_sample, samples_per_cta))
    return fail(ctx, PLAN_EINVAL, "need (1, 1..8), (2, 1), (2, 2), (2, 4) or (4, 1)");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, cudaStreamSynchronize(ctx->internal));
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();   // their layout buffers stay in the arena until plan_destroy
  ctx->tune_wps = warps_per_sample;
  ctx->tune_spc = samples_per_cta;
  return PLAN_OK;
}

int plan_set_persistent(plan_ctx* ctx, int mode) {
  if (!ctx) return PLAN_EINVAL;
  if (mode != PLAN_PERSIST_AUTO && mode != PLAN_PERSIST_OFF && mode != PLAN_PERSIST_ON)
    return fail(ctx, PLAN_EINVAL, "mode must be PLAN_PERSIST_AUTO, _OFF or _ON");
  CU(ctx, cudaSetDevice(ctx->device));
  CU(ctx, cudaStreamSynchronize(ctx->internal));
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  ctx->persist = mode;
  return PLAN_OK;
}

int plan_autotune(plan_ctx* ctx, const plan_scene* scene, int B, int* wps_out, int* spc_out,
                  void* stream) {
  if (!ctx) return PLAN_EINVAL;
  if (!scene || !wps_out || !spc_out) return fail(ctx, PLAN_EINVAL, "NULL argument");
  if (B < 1 || B > ctx->cfg.max_samples) return fail(ctx, PLAN_ECAPACITY, "B out of range");
  TRY(check_scene(ctx, scene, 0));
  *wps_out = 0;
  *spc_out = 0;
  if (ctx->cfg.prec != PLAN_PREC_FP32) return PLAN_OK;
  const char* cache = std::getenv("PLAN_TUNE_CACHE");
  if (cache && *cache) {
    if (FILE* f = std::fopen(cache, "r")) {
      int n, m, N, b, w, sp;
      double ms;
      int found_w = 0, found_s = 0;
      while (std::fscanf(f, "%d %d %d %d %d %d %lf", &n, &m, &N, &b, &w, &sp, &ms) == 7)
        if (n == ctx->cfg.n_coef && m == ctx->cfg.m && N == scene->n_obs && b == B &&
            fused_shape_ok(w, sp)) { found_w = w; found_s = sp; }
      std::fclose(f);
      if (found_w) {
        TRY(plan_set_tuning(ctx, found_w, found_s));
        *wps_out = found_w;
        *spc_out = found_s;
        return PLAN_OK;
      }
    }
  }
  CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // samples from the uniform first-iteration distribution
  plan_cem_state st{};
  st.fresh = 1;
  st.seed = 0x5eedull;
  TRY(plan_sample(ctx, scene, nullptr, nullptr, 1, 1, st.seed, 0, B, ctx->p, stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(ctx, cudaEventCreate(&e0));
  CU(ctx, cudaEventCreate(&e1));
  const int cand[][2] = {{1, 1}, {1, 2}, {1, 4}, {1, 5}, {1, 6}, {1, 7}, {1, 8},
                        {2, 1}, {2, 2}, {2, 4}, {4, 1}};
  const int save_w = ctx->tune_wps, save_s = ctx->tune_spc;
  int best_w = 0, best_s = 0;
  float best = 1e30f;
  std::vector<int> Bv{B};
  int st_code = PLAN_OK;
  for (const auto& cnd : cand) {
    ctx->tune_wps = cnd[0];
    ctx->tune_spc = cnd[1];
    st_code = upload(ctx, ctx->tr, scene, 1, &Bv, s, nullptr);
    if (st_code != PLAN_OK) break;
    const int nt = n_tiles_of(Bv, cnd[1]);
    float times[3];
    cudaError_t ce =
        run_solve(ctx, ctx->tr, ctx->tr, nt, B, 1, ctx->p, nullptr, ctx->r, ctx->cu, nullptr, s);
    for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      ce = run_solve(ctx, ctx->tr, ctx->tr, nt, B, 1, ctx->p, nullptr, ctx->r, ctx->cu, nullptr, s);
      cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&times[rep], e0, e1);
    }
    if (ce != cudaSuccess) {
      st_code = fail(ctx, PLAN_ECUDA, "autotune launch failed: %s", cudaGetErrorString(ce));
      break;
    }
    std::sort(times, times + 3);
    if (times[1] < best) { best = times[1]; best_w = cnd[0]; best_s = cnd[1]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune_wps = save_w;
  ctx->tune_spc = save_s;
  if (st_code != PLAN_OK) return st_code;
  TRY(plan_set_tuning(ctx, best_w, best_s));
  if (cache && *cache) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "%d %d %d %d %d %d %.6f\n", ctx->cfg.n_coef, ctx->cfg.m, scene->n_obs, B, best_w,
                   best_s, double(best));
      std::fclose(f);
    }
  }
  *wps_out = best_w;
  *spc_out = best_s;
  return PLAN_OK;
}

int plan_advance(const plan_config* cfg, const plan_scene* in, const double* xi, int steps,
                 plan_scene* out, plan_obstacle* out_obs) {
  if (!cfg || !in || !xi || !out || (in->n_obs > 0 && (!in->obs || !out_obs)))
    return fail(nullptr, PLAN_EINVAL, "NULL argument");
  if (cfg->m < 2 || cfg->n_coef < 2 || cfg->n_coef > kMaxCoef || !(cfg->dt > 0))
    return fail(nullptr, PLAN_EINVAL, "invalid m, n_coef or dt");
  if (steps < 0 || steps >= cfg->m) return fail(nullptr, PLAN_EINVAL, "steps must be in [0, m)");
  // Bernstein polynomial of degree n-1 and its first two derivatives at
  // tau = steps / (m - 1), through de Casteljau differences of the coefficients
  const int n = cfg->n_coef, deg = n - 1;
  const double tf = (cfg->m - 1) * cfg->dt, tau = double(steps) / (cfg->m - 1);
  double st[6];
  for (int axis = 0; axis < 2; ++axis) {
    const double* c = xi + axis * n;
    double d0[kMaxCoef], d1[kMaxCoef], d2[kMaxCoef];
    for (int k = 0; k < n; ++k) d0[k] = c[k];
    for (int k = 0; k + 1 < n; ++k) d1[k] = deg * (c[k + 1] - c[k]);
    for (int k = 0; k + 2 < n; ++k) d2[k] = (deg - 1) * (d1[k + 1] - d1[k]);
    auto casteljau = [&](double* b, int len) {
      for (int r = 1; r < len; ++r)
        for (int k = 0; k + r < len; ++k) b[k] = (1.0 - tau) * b[k] + tau * b[k + 1];
      return len > 0 ? b[0] : 0.0;
    };
    st[axis] = casteljau(d0, n);
    st[2 + axis] = casteljau(d1, n - 1) / tf;
    st[4 + axis] = n > 2 ? casteljau(d2, n - 2) / (tf * tf) : 0.0;
  }
  const double t = steps * cfg->dt;
  plan_scene o = *in;
  o.ego.x = 0.0;
  o.ego.y = st[1];
  o.ego.vx = st[2];
  o.ego.vy = st[3];
  o.ego.ax = st[4];
  o.ego.ay = st[5];
  for (int i = 0; i < in->n_obs; ++i) {
    plan_obstacle ob = in->obs[i];
    ob.x0 = ob.x0 + ob.vx * t - st[0];
    ob.y0 = ob.y0 + ob.vy * t;
    out_obs[i] = ob;
  }
  o.obs = in->n_obs > 0 ? out_obs : nullptr;
  o.road_origin = in->road_origin + st[0];   // same knots, frame moved with the ego
  *out = o;
  return PLAN_OK;
}

}  // extern "C"

// Serving loop: continuous batching of planning requests (one MPC cycle of
// Alg. 1 each) from many driving scenes.
//
// A scheduler thread owns a pool of executors.  An executor is a planner
// context for one horizon m (its own constants, arena and stream).  Pending
// requests are admitted into a wave of an idle executor of their horizon while
// its sample and scene capacity allow; a new executor is created while the
// device-memory budget and the executor limit allow.  Waves of different
// executors run concurrently on the device.  Each request belongs to an
// episode whose sampling distribution (mu, Sigma, step) stays in a device
// table between cycles: a wave gathers the states of continuing episodes
// from the table, runs Alg. 1 and scatters the final states back.  A host
// callback on the executor's stream marks the wave done; the scheduler then
// completes its tickets.  No wait is unbounded: the scheduler sleeps on a
// condition variable with a short timeout and plan_poll takes a timeout.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

using namespace plan;

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  plan_scene scene{};
  std::vector<plan_obstacle> obs;
  std::vector<plan_road_knot> road;
  int B = 0, m = 0;
  uint64_t episode = 0, seed = 0;
  int fresh = 0;
  int row = -1;          // episode row in the device table
  double t_submit = 0;
};

struct Ticket {
  bool done = false;
  int status = PLAN_OK;
  plan_result res{};
  double t_submit = 0, t_done = 0;
};

struct Executor {
  int m = 0;
  plan_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  DevCem* h_init = nullptr;      // pinned, [cap_scenes]
  DevCem* h_res = nullptr;       // pinned, [cap_scenes]
  std::vector<Request> wave;
  std::atomic<bool> done{false};
  bool busy = false;
  size_t bytes = 0;
  plan_server* srv = nullptr;
};

}  // namespace

struct plan_server {
  plan_config base{};
  int max_exec = 0, max_episodes = 0;
  size_t budget = 0, bytes_used = 0;
  int device = 0;
  DevCem* d_table = nullptr;
  std::unordered_map<uint64_t, int> ep_row;
  std::vector<int> free_rows;
  std::mutex mu;
  std::condition_variable cv;        // scheduler wake-ups
  std::condition_variable cv_done;   // ticket completions
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Ticket> tickets;
  std::deque<uint64_t> done_q;       // completed tickets in completion order
  uint64_t next_ticket = 1;
  std::vector<std::unique_ptr<Executor>> execs;
  std::thread worker;
  bool stop = false;
  std::string err;
  uint64_t n_waves = 0, n_done = 0, max_wave = 0;
};

namespace {

void CUDART_CB on_wave_done(void* arg) {
  // runs on a CUDA callback thread: no CUDA calls, no blocking lock
  Executor* e = static_cast<Executor*>(arg);
  e->done.store(true);
  e->srv->cv.notify_all();
}

// A new executor for horizon m (called without the lock: plan_init allocates
// and builds constants; the caller adds it to the server under the lock).
int make_executor(plan_server* s, int m, std::unique_ptr<Executor>* out) {
  plan_config cfg = s->base;
  cfg.m = m;
  plan_ctx* ctx = nullptr;
  int st = plan_init(&cfg, &ctx);
  if (st != PLAN_OK) return st;
  // a fixed kernel shape per executor: a scene's arithmetic must not depend on
  // how many other samples share its wave.  Executors launch one CTA per tile:
  // waves of several executors share the device, and a persistent grid would
  // hold every SM it fits on until its last sample is done, keeping the other
  // waves' CTAs out (both launch forms give the same bits)
  if (cfg.prec == PLAN_PREC_FP32) {
    st = m > 128 ? plan_set_tuning(ctx, 2, 2) : plan_set_tuning(ctx, 1, 4);
    if (st == PLAN_OK) st = plan_set_persistent(ctx, PLAN_PERSIST_OFF);
    if (st != PLAN_OK) {
      plan_destroy(ctx);
      return st;
    }
  }
  auto e = std::make_unique<Executor>();
  e->m = m;
  e->ctx = ctx;
  e->srv = s;
  e->bytes = ctx_bytes(ctx);
  const size_t nb = sizeof(DevCem) * cfg.max_scenes;
  if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&e->h_init), nb, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&e->h_res), nb, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    if (e->stream) cudaStreamDestroy(e->stream);
    if (e->h_init) cudaFreeHost(e->h_init);
    if (e->h_res) cudaFreeHost(e->h_res);
    plan_destroy(ctx);
    return PLAN_ENOMEM;
  }
  *out = std::move(e);
  return PLAN_OK;
}

// Complete the tickets of a finished wave (caller holds the lock).
void finalize(plan_server* s, Executor* e) {
  const double t = now_us();
  const int d_p = 2 * s->base.n_seg + 2 * s->base.goal, nx = 2 * s->base.n_coef;
  for (size_t i = 0; i < e->wave.size(); ++i) {
    const Request& r = e->wave[i];
    Ticket& tk = s->tickets[r.ticket];
    const DevCem& c = e->h_res[i];
    std::memset(&tk.res, 0, sizeof tk.res);
    for (int a = 0; a < d_p; ++a) tk.res.p[a] = c.best_p[a];
    for (int a = 0; a < nx; ++a) tk.res.xi[a] = c.best_xi[a];
    tk.res.cost = c.best_cost;
    tk.res.resid = c.best_r;
    tk.res.cu = c.best_cu;
    tk.res.index = c.best_index;
    tk.status = std::isfinite(c.best_cost) ? PLAN_OK : PLAN_ENONFINITE;
    tk.t_done = t;
    tk.done = true;
    ++s->n_done;
    s->done_q.push_back(e->wave[i].ticket);
  }
  e->wave.clear();
  e->busy = false;
  e->done.store(false);
  s->cv_done.notify_all();
}

// Move pending requests of the executor's horizon into its wave and mark it
// busy (caller holds the lock).  Returns the wave's size.
int take_wave(plan_server* s, Executor* e) {
  const int cap_s = s->base.max_scenes, cap_b = s->base.max_samples;
  int samples = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && int(e->wave.size()) < cap_s;) {
    if (it->m == e->m && samples + it->B <= cap_b) {
      samples += it->B;
      e->wave.push_back(std::move(*it));
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
  if (!e->wave.empty()) e->busy = true;
  return int(e->wave.size());
}

// Upload and launch a taken wave (called without the lock: it reads only the
// executor's own wave and buffers; waves of different executors hold
// different episodes, so their table rows do not overlap).
int run_wave(plan_server* s, Executor* e) {
  const int S = int(e->wave.size());
  std::vector<plan_scene> scenes(S);
  std::vector<int> B(S), gather(S), scatter(S);
  int st = PLAN_OK;
  for (int i = 0; i < S && st == PLAN_OK; ++i) {
    const Request& r = e->wave[i];
    scenes[i] = r.scene;
    scenes[i].obs = r.obs.empty() ? nullptr : r.obs.data();
    scenes[i].road = r.road.empty() ? nullptr : r.road.data();
    B[i] = r.B;
    plan_cem_state cs{};
    cs.seed = r.seed;
    cs.fresh = 1;
    st = ctx_make_state(e->ctx, &cs, r.scene.n_lanes, r.scene.lane_width, r.scene.ego.x,
                        &e->h_init[i]);
    gather[i] = r.fresh ? -1 : r.row;
    scatter[i] = r.row;
  }
  if (st == PLAN_OK)
    st = ctx_wave(e->ctx, scenes.data(), B.data(), S, e->h_init, gather.data(), scatter.data(),
                  s->d_table, e->h_res, e->stream);
  if (st == PLAN_OK && cudaLaunchHostFunc(e->stream, on_wave_done, e) != cudaSuccess) {
    cudaGetLastError();
    st = PLAN_ECUDA;
  }
  return st;
}

// Book a launched wave, or fail its tickets (caller holds the lock).
void post_wave(plan_server* s, Executor* e, int st) {
  if (st != PLAN_OK) {
    const double t = now_us();
    for (auto& r : e->wave) {
      Ticket& tk = s->tickets[r.ticket];
      tk.status = st;
      tk.done = true;
      tk.t_done = t;
      s->done_q.push_back(r.ticket);
    }
    s->err = ctx_error(e->ctx);
    e->wave.clear();
    e->busy = false;
    s->cv_done.notify_all();
    return;
  }
  ++s->n_waves;
  s->max_wave = std::max<uint64_t>(s->max_wave, uint64_t(e->wave.size()));
}

// Fail the pending requests of horizon m (no executor could be made for it).
void fail_pending(plan_server* s, int m, int st) {
  const double t = now_us();
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    if (it->m == m) {
      Ticket& tk = s->tickets[it->ticket];
      tk.status = st;
      tk.done = true;
      tk.t_done = t;
      s->done_q.push_back(it->ticket);
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
  s->cv_done.notify_all();
}

// The scheduler thread.  It holds the lock only to pick work and to book it:
// a wave's uploads and launches and the creation of an executor run unlocked,
// so that submissions and polls are not held up behind CUDA calls.
void scheduler(plan_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    for (auto& e : s->execs)
      if (e->busy && e->done.load()) finalize(s, e.get());
    // admit pending requests, oldest first, one wave or one new executor at a
    // time (the queue may change while unlocked: rescan after each)
    while (!s->stop) {
      Executor* idle = nullptr;
      int want_m = -1;
      std::vector<int> tried;
      for (const Request& r : s->pending) {
        if (std::find(tried.begin(), tried.end(), r.m) != tried.end()) continue;
        tried.push_back(r.m);
        for (auto& e : s->execs)
          if (!e->busy && e->m == r.m) { idle = e.get(); break; }
        if (idle) break;
        if (want_m < 0 && int(s->execs.size()) < s->max_exec) {
          // admission by memory: estimate from an executor of any horizon
          const size_t est = s->execs.empty() ? 0 : s->execs.front()->bytes;
          if (s->bytes_used + est <= s->budget) want_m = r.m;
        }
      }
      if (idle) {
        if (take_wave(s, idle) == 0) break;
        lk.unlock();
        const int st = run_wave(s, idle);
        lk.lock();
        post_wave(s, idle, st);
        continue;
      }
      if (want_m >= 0) {
        lk.unlock();
        std::unique_ptr<Executor> e;
        const int st = make_executor(s, want_m, &e);
        lk.lock();
        if (st == PLAN_OK) {
          s->bytes_used += e->bytes;
          s->execs.push_back(std::move(e));
          continue;
        }
        // no more executors; requests of a horizon without one cannot run
        s->max_exec = int(s->execs.size());
        s->err = "could not create an executor";
        bool have = false;
        for (auto& x : s->execs) have |= x->m == want_m;
        if (!have) fail_pending(s, want_m, st);
        continue;
      }
      break;
    }
    bool busy = false;
    for (auto& e : s->execs) busy |= e->busy;
    if (busy) s->cv.wait_for(lk, std::chrono::microseconds(200));
    else s->cv.wait_for(lk, std::chrono::milliseconds(20));
  }
}

int fail_srv(plan_server* s, int code, const char* msg) {
  if (s) s->err = msg;
  set_unbound_error(msg);
  return code;
}

}  // namespace

extern "C" {

int plan_server_create(const plan_config* cfg, int max_executors, size_t device_budget,
                       int max_episodes, plan_server** out) {
  if (!out) return PLAN_EINVAL;
  *out = nullptr;
  if (!cfg || max_executors < 1 || max_episodes < 1 || device_budget == 0)
    return fail_srv(nullptr, PLAN_EINVAL, "need cfg, max_executors >= 1, max_episodes >= 1, a budget");
  // validate the configuration once (and learn the executor size)
  plan_ctx* probe = nullptr;
  int st = plan_init(cfg, &probe);
  if (st != PLAN_OK) return st;
  const size_t per = ctx_bytes(probe);
  plan_destroy(probe);
  if (per > device_budget) return fail_srv(nullptr, PLAN_ENOMEM, "budget below one executor");
  auto* s = new plan_server();
  s->base = *cfg;
  s->max_exec = max_executors;
  s->budget = device_budget;
  s->max_episodes = max_episodes;
  cudaGetDevice(&s->device);
  if (cudaMalloc(&s->d_table, sizeof(DevCem) * max_episodes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail_srv(nullptr, PLAN_ENOMEM, "episode table allocation failed");
  }
  s->bytes_used = sizeof(DevCem) * max_episodes;
  for (int i = max_episodes - 1; i >= 0; --i) s->free_rows.push_back(i);
  s->worker = std::thread(scheduler, s);
  *out = s;
  return PLAN_OK;
}

int plan_server_destroy(plan_server* s) {
  if (!s) return PLAN_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& e : s->execs) {
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->stream) cudaStreamDestroy(e->stream);
    if (e->h_init) cudaFreeHost(e->h_init);
    if (e->h_res) cudaFreeHost(e->h_res);
    plan_destroy(e->ctx);
  }
  cudaFree(s->d_table);
  delete s;
  return PLAN_OK;
}

int plan_submit(plan_server* s, const plan_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return fail_srv(s, PLAN_EINVAL, "NULL argument");
  const int m = req->m > 0 ? req->m : s->base.m;
  if (req->B < 1 || req->B > s->base.max_samples)
    return fail_srv(s, PLAN_ECAPACITY, "B outside [1, max_samples]");
  if (m < 8 || m > 256) return fail_srv(s, PLAN_EINVAL, "horizon m must be in [8, 256]");
  const plan_scene& sc = req->scene;
  if (sc.n_obs < 0 || sc.n_obs > s->base.max_obs)
    return fail_srv(s, PLAN_ECAPACITY, "n_obs exceeds max_obs");
  if (sc.n_obs > 0 && !sc.obs) return fail_srv(s, PLAN_EINVAL, "obs is NULL");
  if (sc.n_lanes < 1 || !(sc.lane_width > 0)) return fail_srv(s, PLAN_EINVAL, "invalid lanes");
  if (const char* why = road_invalid(sc, s->base.lane_margin)) return fail_srv(s, PLAN_EINVAL, why);
  Request r;
  r.scene = sc;
  r.obs.assign(sc.obs, sc.obs + sc.n_obs);
  r.road.assign(sc.road, sc.road + sc.n_road);
  r.B = req->B;
  r.m = m;
  r.episode = req->episode;
  r.seed = req->seed;
  r.t_submit = now_us();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->ep_row.find(req->episode);
    if (it == s->ep_row.end()) {
      if (s->free_rows.empty()) return fail_srv(s, PLAN_ECAPACITY, "episode table full");
      r.row = s->free_rows.back();
      s->free_rows.pop_back();
      s->ep_row[req->episode] = r.row;
      r.fresh = 1;
    } else {
      r.row = it->second;
      r.fresh = req->fresh ? 1 : 0;
    }
    r.ticket = s->next_ticket++;
    Ticket tk;
    tk.t_submit = r.t_submit;
    s->tickets[r.ticket] = tk;
    *ticket = r.ticket;
    s->pending.push_back(std::move(r));
  }
  s->cv.notify_all();
  return PLAN_OK;
}

int plan_poll(plan_server* s, uint64_t ticket, plan_result* out, double* latency_us,
              int timeout_us) {
  if (!s) return PLAN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return fail_srv(s, PLAN_EINVAL, "unknown ticket");
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  while (!it->second.done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = s->tickets.find(ticket);
      if (!it->second.done) return PLAN_ETIMEOUT;
      break;
    }
    it = s->tickets.find(ticket);
  }
  const Ticket tk = it->second;
  s->tickets.erase(it);
  if (out) *out = tk.res;
  if (latency_us) *latency_us = tk.t_done - tk.t_submit;
  return tk.status;
}

int plan_poll_any(plan_server* s, uint64_t* ticket, plan_result* out, double* latency_us,
                  int timeout_us) {
  if (!s || !ticket) return PLAN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  for (;;) {
    // tickets already taken by plan_poll are stale entries: drop them
    while (!s->done_q.empty() && s->tickets.find(s->done_q.front()) == s->tickets.end())
      s->done_q.pop_front();
    if (!s->done_q.empty()) break;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      while (!s->done_q.empty() && s->tickets.find(s->done_q.front()) == s->tickets.end())
        s->done_q.pop_front();
      if (s->done_q.empty()) return PLAN_ETIMEOUT;
      break;
    }
  }
  const uint64_t id = s->done_q.front();
  s->done_q.pop_front();
  auto it = s->tickets.find(id);
  const Ticket tk = it->second;
  s->tickets.erase(it);
  *ticket = id;
  if (out) *out = tk.res;
  if (latency_us) *latency_us = tk.t_done - tk.t_submit;
  return tk.status;
}

int plan_end_episode(plan_server* s, uint64_t episode) {
  if (!s) return PLAN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ep_row.find(episode);
  if (it == s->ep_row.end()) return fail_srv(s, PLAN_EINVAL, "unknown episode");
  for (const Request& r : s->pending)
    if (r.episode == episode) return fail_srv(s, PLAN_ESTATE, "episode has a pending request");
  for (auto& e : s->execs)
    for (const Request& r : e->wave)
      if (r.episode == episode) return fail_srv(s, PLAN_ESTATE, "episode has a request in flight");
  s->free_rows.push_back(it->second);
  s->ep_row.erase(it);
  return PLAN_OK;
}

int plan_server_info(plan_server* s, plan_server_stats* out) {
  if (!s || !out) return PLAN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof *out);
  out->executors = int(s->execs.size());
  for (auto& e : s->execs) out->busy += e->busy ? 1 : 0;
  out->pending = int(s->pending.size());
  out->waves = s->n_waves;
  out->completed = s->n_done;
  out->max_wave = int(s->max_wave);
  out->device_bytes = s->bytes_used;
  return PLAN_OK;
}

}  // extern "C"

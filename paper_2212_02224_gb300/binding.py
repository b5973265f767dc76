"""ctypes binding of include/plan.h: the same names, argument marshalling only.

Every step of the planner runs in the CUDA library; this module only converts
Python objects to the C structs and raw pointers the C ABI takes.  It raises
if the library has not been built -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libplan.so")

PLAN_OK = 0
PLAN_EINVAL = -1
PLAN_ENOMEM = -2
PLAN_ECAPACITY = -3
PLAN_ETIMEOUT = -4
PLAN_ECUDA = -5
PLAN_ESTATE = -6
PLAN_ENONFINITE = -7

PLAN_PREC_FP64 = 0
PLAN_PREC_FP32 = 1
PLAN_PREC_TF32 = 2
PLAN_PREC_BF16 = 3
PLAN_PREC_TF32X3 = 4
PLAN_MAX_DP = 10
PRECISIONS = {"fp64": PLAN_PREC_FP64, "fp32": PLAN_PREC_FP32, "tf32": PLAN_PREC_TF32,
              "bf16": PLAN_PREC_BF16, "tf32x3": PLAN_PREC_TF32X3}


class PlanConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "m", "n_coef", "n_seg", "inner_iters", "outer_iters", "n_elite_c", "n_elite", "prec",
        "max_obs", "max_samples", "max_scenes", "goal")] + [(n, ctypes.c_double) for n in (
        "dt", "rho", "kp_lat", "kv_lat", "kp_lon", "gamma", "eta", "cov_eps", "v_min", "v_max",
        "a_max", "kappa_max", "c_max", "lane_margin", "v_des_lo", "v_des_hi")]


class PlanEgo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("x", "y", "vx", "vy", "ax", "ay")]


class PlanObstacle(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("x0", "y0", "vx", "vy", "a", "b")]


class PlanRoadKnot(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("s", "kappa", "lb", "ub")]


class PlanScene(ctypes.Structure):
    _fields_ = [("ego", PlanEgo), ("n_lanes", ctypes.c_int), ("lane_width", ctypes.c_double),
                ("kappa_road", ctypes.c_double), ("n_obs", ctypes.c_int),
                # const plan_obstacle* / const plan_road_knot*: set from the
                # address of a float64 buffer with the same row layout
                ("obs", ctypes.c_void_p), ("n_road", ctypes.c_int),
                ("road", ctypes.c_void_p), ("road_origin", ctypes.c_double)]


class PlanCemState(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double * PLAN_MAX_DP), ("sigma", ctypes.c_double * (PLAN_MAX_DP ** 2)),
                ("seed", ctypes.c_uint64), ("episode_step", ctypes.c_uint64),
                ("fresh", ctypes.c_int), ("reserved0", ctypes.c_int)]


class PlanRequest(ctypes.Structure):
    _fields_ = [("scene", PlanScene), ("B", ctypes.c_int), ("m", ctypes.c_int),
                ("episode", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("fresh", ctypes.c_int), ("reserved0", ctypes.c_int)]


class PlanServerStats(ctypes.Structure):
    _fields_ = [("executors", ctypes.c_int), ("busy", ctypes.c_int), ("pending", ctypes.c_int),
                ("max_wave", ctypes.c_int), ("waves", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("device_bytes", ctypes.c_size_t)]


class PlanResult(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double * PLAN_MAX_DP), ("xi", ctypes.c_double * 32),
                ("cost", ctypes.c_double), ("resid", ctypes.c_double), ("cu", ctypes.c_double),
                ("index", ctypes.c_int), ("reserved0", ctypes.c_int)]


EXPORTS = ("plan_init", "plan_destroy", "plan_status_str", "plan_last_error", "plan_solve",
           "plan_solve_batch", "plan_upload_scenes", "plan_set_state", "plan_get_state",
           "plan_step_resident", "plan_get_result", "plan_step", "plan_select_elites",
           "plan_update_distribution", "plan_sample", "plan_set_tuning", "plan_autotune",
           "plan_solve_fp64_noalloc", "plan_advance", "plan_server_create", "plan_server_destroy",
           "plan_submit", "plan_poll", "plan_poll_any", "plan_end_episode", "plan_server_info",
           "plan_qp_forward", "plan_qp_backward", "plan_probe_alu", "plan_probe_wait_timeout",
           "plan_probe_tc_wide", "plan_set_persistent")

_lib = None


class PlanError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_str(status)} ({status}): {msg}")
        self.status = status


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libplan.so (built by build.py, or the file named by the environment
    variable PLAN_LIBRARY); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PLAN_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"planner CUDA library not built: {path} is missing "
                           "(run paper_2212_02224_gb300/build.py)")
    lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    P, I, D, V, U64 = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64
    sig = {
        "plan_init": (I, [P(PlanConfig), P(V)]),
        "plan_destroy": (I, [V]),
        "plan_status_str": (ctypes.c_char_p, [I]),
        "plan_last_error": (I, [V, ctypes.c_char_p, ctypes.c_size_t]),
        "plan_solve": (I, [V, P(PlanScene), V, I, V, V, V, V, V]),
        "plan_solve_batch": (I, [V, P(PlanScene), P(I), I, V, V, V, V, V, V]),
        "plan_upload_scenes": (I, [V, P(PlanScene), I, V]),
        "plan_set_state": (I, [V, I, P(PlanCemState), V]),
        "plan_get_state": (I, [V, I, P(PlanCemState), V]),
        "plan_step_resident": (I, [V, P(I), I, V]),
        "plan_get_result": (I, [V, I, P(PlanResult), V]),
        "plan_step": (I, [V, P(PlanScene), P(PlanCemState), I, P(PlanResult), V]),
        "plan_select_elites": (I, [V, V, V, I, I, I, V, V]),
        "plan_update_distribution": (I, [V, V, V, I, V, V, V]),
        "plan_sample": (I, [V, P(PlanScene), V, V, I, I, U64, U64, I, V, V]),
        "plan_set_tuning": (I, [V, I, I]),
        "plan_set_persistent": (I, [V, I]),
        "plan_autotune": (I, [V, P(PlanScene), I, P(I), P(I), V]),
        "plan_solve_fp64_noalloc": (I, [P(PlanConfig), P(PlanScene), V, I, V, V, V, V]),
        "plan_advance": (I, [P(PlanConfig), P(PlanScene), P(D), I, P(PlanScene), P(PlanObstacle)]),
        "plan_server_create": (I, [P(PlanConfig), I, ctypes.c_size_t, I, P(V)]),
        "plan_server_destroy": (I, [V]),
        "plan_submit": (I, [V, P(PlanRequest), P(U64)]),
        "plan_poll": (I, [V, U64, P(PlanResult), P(D), I]),
        "plan_poll_any": (I, [V, P(U64), P(PlanResult), P(D), I]),
        "plan_end_episode": (I, [V, U64]),
        "plan_server_info": (I, [V, P(PlanServerStats)]),
        "plan_qp_forward": (I, [V, V, V, I, V, V]),
        "plan_qp_backward": (I, [V, V, I, V, V, V]),
        "plan_probe_alu": (I, [P(D), V]),
        "plan_probe_wait_timeout": (I, [I, V]),
        "plan_probe_tc_wide": (I, [I, I, P(D), V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_str(status: int) -> str:
    try:
        return load().plan_status_str(status).decode()
    except RuntimeError:
        return str(status)


def last_error(ctx) -> str:
    buf = ctypes.create_string_buffer(512)
    load().plan_last_error(ctx, buf, 512)
    return buf.value.decode()


def check(status: int, ctx=None) -> None:
    if status != PLAN_OK:
        raise PlanError(status, last_error(ctx))


# ----------------------------------------------------------------------------- marshalling

def make_config(prm, prec: int, max_obs: int, max_samples: int, max_scenes: int = 1) -> PlanConfig:
    """PlanConfig from any object with the planner's parameter attributes."""
    c = PlanConfig()
    for name in ("m", "n_coef", "n_seg", "inner_iters", "outer_iters", "n_elite_c", "n_elite"):
        setattr(c, name, int(getattr(prm, name)))
    for name in ("dt", "rho", "kp_lat", "kv_lat", "kp_lon", "gamma", "eta", "cov_eps", "v_min",
                 "v_max", "a_max", "kappa_max", "c_max", "lane_margin", "v_des_lo", "v_des_hi"):
        setattr(c, name, float(getattr(prm, name)))
    c.prec = int(prec)
    c.max_obs, c.max_samples, c.max_scenes = int(max_obs), int(max_samples), int(max_scenes)
    c.goal = int(bool(getattr(prm, "goal", False)))
    return c


def _rows(a, width):
    """Contiguous float64 (rows x width) view of a, copied only when needed."""
    if isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous:
        return a.reshape(-1, width)
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, width))


def make_scenes(scenes):
    """(PlanScene array, keep-alive list) from objects with ego / n_lanes /
    lane_width / kappa_road / obstacles (N x 6 rows x0, y0, vx, vy, a, b)."""
    arr = (PlanScene * len(scenes))()
    keep = []
    for i, sc in enumerate(scenes):
        e = sc.ego
        arr[i].ego = PlanEgo(float(e[0]), float(e[1]), float(e[2]), float(e[3]), float(e[4]),
                             float(e[5]))
        arr[i].n_lanes = int(sc.n_lanes)
        arr[i].lane_width = float(sc.lane_width)
        arr[i].kappa_road = float(sc.kappa_road)
        # obstacle rows and road knots are passed straight from float64 buffers
        # laid out like plan_obstacle / plan_road_knot
        ob = _rows(sc.obstacles, 6)
        arr[i].n_obs = ob.shape[0]
        if ob.shape[0]:
            keep.append(ob)
            arr[i].obs = ob.ctypes.data
        else:
            arr[i].obs = None
        road = getattr(sc, "road", None)
        road = _rows(road, 4) if road is not None and len(road) else None
        arr[i].n_road = 0 if road is None else road.shape[0]
        if road is not None:
            keep.append(road)
            arr[i].road = road.ctypes.data
        else:
            arr[i].road = None
        arr[i].road_origin = float(getattr(sc, "road_origin", 0.0))
    keep.append(arr)
    return arr, keep


def make_state(d_p: int, mu=None, sigma=None, seed: int = 0, step: int = 0, fresh=None) -> PlanCemState:
    st = PlanCemState()
    st.seed, st.episode_step = int(seed), int(step)
    st.fresh = int(mu is None if fresh is None else fresh)
    if mu is not None:
        for a in range(d_p):
            st.mu[a] = float(mu[a])
            for b in range(d_p):
                st.sigma[a * PLAN_MAX_DP + b] = float(sigma[a][b])
    return st


def state_arrays(st: PlanCemState, d_p: int):
    mu = [st.mu[a] for a in range(d_p)]
    sigma = [[st.sigma[a * PLAN_MAX_DP + b] for b in range(d_p)] for a in range(d_p)]
    return mu, sigma


# ----------------------------------------------------------------------------- entry points

def plan_init(cfg: PlanConfig):
    ctx = ctypes.c_void_p()
    check(load().plan_init(ctypes.byref(cfg), ctypes.byref(ctx)), None)
    return ctx


def plan_destroy(ctx) -> None:
    check(load().plan_destroy(ctx), None)


def plan_solve(ctx, scene, p_ptr: int, B: int, xi_ptr, r_ptr: int, cu_ptr: int, status_ptr=None,
               stream: int = 0):
    arr, keep = make_scenes([scene])
    check(load().plan_solve(ctx, arr, p_ptr, B, xi_ptr, r_ptr, cu_ptr, status_ptr, stream), ctx)


def plan_solve_batch(ctx, scenes, Bs, p_ptr: int, xi_ptr, r_ptr: int, cu_ptr: int, status_ptr=None,
                     stream: int = 0):
    arr, keep = make_scenes(scenes)
    b = (ctypes.c_int * len(Bs))(*[int(x) for x in Bs])
    check(load().plan_solve_batch(ctx, arr, b, len(Bs), p_ptr, xi_ptr, r_ptr, cu_ptr, status_ptr,
                                  stream), ctx)


def plan_upload_scenes(ctx, scenes, stream: int = 0):
    arr, keep = make_scenes(scenes)
    check(load().plan_upload_scenes(ctx, arr, len(scenes), stream), ctx)


def plan_set_state(ctx, slot: int, st: PlanCemState, stream: int = 0):
    check(load().plan_set_state(ctx, slot, ctypes.byref(st), stream), ctx)


def plan_get_state(ctx, slot: int, stream: int = 0) -> PlanCemState:
    st = PlanCemState()
    check(load().plan_get_state(ctx, slot, ctypes.byref(st), stream), ctx)
    return st


def plan_step_resident(ctx, Bs, stream: int = 0):
    b = (ctypes.c_int * len(Bs))(*[int(x) for x in Bs])
    check(load().plan_step_resident(ctx, b, len(Bs), stream), ctx)


def plan_get_result(ctx, slot: int, stream: int = 0) -> PlanResult:
    out = PlanResult()
    check(load().plan_get_result(ctx, slot, ctypes.byref(out), stream), ctx)
    return out


def plan_step(ctx, scene, st: PlanCemState, B: int, stream: int = 0) -> PlanResult:
    arr, keep = make_scenes([scene])
    out = PlanResult()
    check(load().plan_step(ctx, arr, ctypes.byref(st), B, ctypes.byref(out), stream), ctx)
    return out


def plan_select_elites(ctx, r_ptr: int, cu_ptr: int, B: int, n_c: int, q: int, elite_ptr: int,
                       stream: int = 0):
    check(load().plan_select_elites(ctx, r_ptr, cu_ptr, B, n_c, q, elite_ptr, stream), ctx)


def plan_update_distribution(ctx, p_ptr: int, cost_ptr: int, q: int, mu_ptr: int, sigma_ptr: int,
                             stream: int = 0):
    check(load().plan_update_distribution(ctx, p_ptr, cost_ptr, q, mu_ptr, sigma_ptr, stream), ctx)


def plan_sample(ctx, scene, mu, sigma, fresh: int, l: int, seed: int, step: int, B: int, p_ptr: int,
                stream: int = 0):
    arr, keep = make_scenes([scene])
    d = len(mu) if mu is not None else 0
    mu_c = (ctypes.c_double * max(d, 1))(*([float(v) for v in mu] if mu is not None else [0.0]))
    sg_c = (ctypes.c_double * max(d * d, 1))(
        *([float(sigma[a][b]) for a in range(d) for b in range(d)] if sigma is not None else [0.0]))
    check(load().plan_sample(ctx, arr, mu_c, sg_c, int(fresh), int(l), int(seed), int(step), int(B),
                             p_ptr, stream), ctx)


def plan_qp_forward(ctx, p_ptr: int, b0_ptr: int, B: int, xi_ptr: int, stream: int = 0):
    check(load().plan_qp_forward(ctx, p_ptr, b0_ptr, int(B), xi_ptr, stream), ctx)


def plan_qp_backward(ctx, g_ptr: int, B: int, grad_p_ptr: int, grad_b0_ptr, stream: int = 0):
    check(load().plan_qp_backward(ctx, g_ptr, int(B), grad_p_ptr, grad_b0_ptr, stream), ctx)


def plan_probe_alu(stream: int = 0) -> dict:
    """Measured arithmetic ceilings of the current device (see include/plan.h)."""
    out = (ctypes.c_double * 5)()
    check(load().plan_probe_alu(out, stream), None)
    return dict(fp32_tflops=out[0], fp32x2_tflops=out[1], fp64_tflops=out[2],
                rsqrt_tops=out[3], sms=int(out[4]))


def plan_probe_tc_wide(passes: int = 3, iters: int = 200, stream: int = 0) -> dict:
    """SM cycles per Alg. 2 iteration of the tensor-core contractions at
    N = 128 columns (64 samples of the n = 16, m = 200 workload), see
    include/plan.h."""
    out = (ctypes.c_double * 6)()
    check(load().plan_probe_tc_wide(int(passes), int(iters), out, stream), None)
    return dict(forward_cycles=out[0], transposed_n16_cycles=out[1],
                transposed_n128_cycles=out[2], transposed_n16_4acc_cycles=out[3],
                transposed_n128_4acc_cycles=out[4], ctas=int(out[5]))


def plan_probe_wait_timeout(wait_us: int, stream: int = 0) -> int:
    """Run one bounded wait that receives no arrival (see include/plan.h) and
    return its status: PLAN_ETIMEOUT is the expected outcome."""
    return int(load().plan_probe_wait_timeout(int(wait_us), stream))


def plan_set_tuning(ctx, warps_per_sample: int, samples_per_cta: int):
    check(load().plan_set_tuning(ctx, int(warps_per_sample), int(samples_per_cta)), ctx)


PLAN_PERSIST_AUTO, PLAN_PERSIST_OFF, PLAN_PERSIST_ON = 0, 1, 2
_PERSIST = {"auto": PLAN_PERSIST_AUTO, "off": PLAN_PERSIST_OFF, "on": PLAN_PERSIST_ON}


def plan_set_persistent(ctx, mode):
    """mode: "auto", "off", "on" or the PLAN_PERSIST_* value."""
    check(load().plan_set_persistent(ctx, int(_PERSIST.get(mode, mode))), ctx)


def plan_autotune(ctx, scene, B: int, stream: int = 0):
    arr, keep = make_scenes([scene])
    w, s = ctypes.c_int(), ctypes.c_int()
    check(load().plan_autotune(ctx, arr, int(B), ctypes.byref(w), ctypes.byref(s), stream), ctx)
    return w.value, s.value


def plan_solve_fp64_noalloc(cfg: PlanConfig, scene, p_ptr: int, B: int, xi_ptr, r_ptr: int,
                            cu_ptr: int, stream: int = 0):
    """Allocation-free float64 solve (no context; see include/plan.h)."""
    arr, keep = make_scenes([scene])
    check(load().plan_solve_fp64_noalloc(ctypes.byref(cfg), arr, p_ptr, int(B), xi_ptr, r_ptr,
                                         cu_ptr, stream), None)


class SceneView:
    """Plain scene record (ego, n_lanes, lane_width, kappa_road, obstacles,
    road knots, road_origin)."""

    def __init__(self, ego, n_lanes, lane_width, kappa_road, obstacles, road=(), road_origin=0.0):
        self.ego, self.n_lanes, self.lane_width = list(ego), n_lanes, lane_width
        self.kappa_road, self.obstacles = kappa_road, [list(o) for o in obstacles]
        self.road, self.road_origin = [list(k) for k in road], road_origin

    @property
    def n_obs(self):
        return len(self.obstacles)


def plan_advance(cfg: PlanConfig, scene, xi, steps: int):
    """MPC advance (see include/plan.h); returns the next scene as a SceneView."""
    arr, keep = make_scenes([scene])
    n_obs = arr[0].n_obs
    xi_c = (ctypes.c_double * len(xi))(*[float(v) for v in xi])
    out = PlanScene()
    out_obs = (PlanObstacle * max(n_obs, 1))()
    check(load().plan_advance(ctypes.byref(cfg), arr, xi_c, int(steps), ctypes.byref(out),
                              out_obs), None)
    e = out.ego
    obs = [[out_obs[i].x0, out_obs[i].y0, out_obs[i].vx, out_obs[i].vy, out_obs[i].a, out_obs[i].b]
           for i in range(n_obs)]
    return SceneView([e.x, e.y, e.vx, e.vy, e.ax, e.ay], out.n_lanes, out.lane_width,
                     out.kappa_road, obs, getattr(scene, "road", []), out.road_origin)


def plan_server_create(cfg: PlanConfig, max_executors: int, device_budget: int, max_episodes: int):
    srv = ctypes.c_void_p()
    check(load().plan_server_create(ctypes.byref(cfg), int(max_executors), int(device_budget),
                                    int(max_episodes), ctypes.byref(srv)), None)
    return srv


def plan_server_destroy(srv):
    check(load().plan_server_destroy(srv), None)


def plan_submit(srv, scene, B: int, m: int = 0, episode: int = 0, seed: int = 0, fresh: int = 0):
    arr, keep = make_scenes([scene])
    req = PlanRequest()
    req.scene = arr[0]
    req.B, req.m, req.episode, req.seed, req.fresh = int(B), int(m), int(episode), int(seed), int(fresh)
    t = ctypes.c_uint64()
    check(load().plan_submit(srv, ctypes.byref(req), ctypes.byref(t)), None)
    return t.value


def plan_poll(srv, ticket: int, timeout_us: int):
    """(status, PlanResult, latency_us); status PLAN_ETIMEOUT means not ready."""
    out = PlanResult()
    lat = ctypes.c_double()
    st = load().plan_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(out), ctypes.byref(lat),
                          int(timeout_us))
    if st not in (PLAN_OK, PLAN_ETIMEOUT):
        check(st, None)
    return st, out, lat.value


def plan_poll_any(srv, timeout_us: int):
    """(status, ticket, PlanResult, latency_us) of the first completed ticket;
    status PLAN_ETIMEOUT (ticket None) means none completed in time."""
    out = PlanResult()
    lat = ctypes.c_double()
    t = ctypes.c_uint64()
    st = load().plan_poll_any(srv, ctypes.byref(t), ctypes.byref(out), ctypes.byref(lat),
                              int(timeout_us))
    if st == PLAN_ETIMEOUT:
        return st, None, out, 0.0
    if st != PLAN_OK:
        check(st, None)
    return st, t.value, out, lat.value


def plan_end_episode(srv, episode: int):
    check(load().plan_end_episode(srv, ctypes.c_uint64(episode)), None)


def plan_server_info(srv):
    st = PlanServerStats()
    check(load().plan_server_info(srv, ctypes.byref(st)), None)
    return {f: getattr(st, f) for f, _ in PlanServerStats._fields_}

"""Seeded synthetic workloads for the batched lower-level trajectory optimizer.

This module only draws inputs: driving scenes (ego state, lanes, obstacle
vehicles), behavioural-input samples p and the numeric parameters of each
workload.  It holds none of the planner's arithmetic, so both the CUDA path
and the FP64 CPU oracle can be fed from it without sharing any method code.

Random numbers come from SplitMix64 (S. Vigna, public-domain reference
algorithm), used as a counter-based generator: draw i of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15).  Scenes stand in for the paper's
highway-env dense-traffic episodes (Sec. V-A): obstacles are ellipses driving
at constant velocity along lane centres, as in the paper's Fig. 4 caption.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` 64-bit outputs of the SplitMix64 stream `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.pos = 0

    def _raw(self, count: int) -> np.ndarray:
        # counter-based: draw j of this reader is output pos + j of the stream
        with np.errstate(over="ignore"):
            i = np.arange(self.pos + 1, self.pos + count + 1, dtype=np.uint64)
            z = np.uint64(self.seed) + i * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out = z ^ (z >> np.uint64(31))
        self.pos += count
        return out

    def uniform(self, lo: float, hi: float, size: int) -> np.ndarray:
        u = (self._raw(size) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, lo: int, hi_inclusive: int, size: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        u = (self._raw(size) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + np.minimum((u * span).astype(np.int64), span - 1)

    def normal(self, mean: float, std: float, size: int) -> np.ndarray:
        """Box-Muller pairs from two uniforms in (0, 1]."""
        k = (size + 1) // 2
        u1 = 1.0 - self.uniform(0.0, 1.0, k)
        u2 = self.uniform(0.0, 1.0, k)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
        return mean + std * z[:size]


@dataclasses.dataclass
class Scene:
    """One driving scene, in a frame where the ego vehicle starts at x = 0.

    ego: (x, y, vx, vy, ax, ay) at t0, the vector b0 of Eq. (boundary_cond_initial).
    obstacles: (N, 6) rows (x0, y0, vx, vy, a, b) -- constant-velocity ellipses
    with semi-axes a (along x) and b (along y), Table I collision row.
    """

    ego: np.ndarray
    n_lanes: int
    lane_width: float
    kappa_road: float
    obstacles: np.ndarray
    # Road profile along the centre line (Frenet frame: x is arc length):
    # (R, 4) knots (s, kappa, lb, ub), interpolated linearly in x and held
    # constant beyond the ends; lb, ub are the road edges.  Empty: a road of
    # constant curvature kappa_road with edges 0 and n_lanes * lane_width.
    road: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 4)))
    road_origin: float = 0.0     # arc length of x = 0 along the road profile

    @property
    def n_obs(self) -> int:
        return int(self.obstacles.shape[0])

    @property
    def n_road(self) -> int:
        return int(np.asarray(self.road).reshape(-1, 4).shape[0])

    def lane_centres(self) -> np.ndarray:
        return (np.arange(self.n_lanes) + 0.5) * self.lane_width


@dataclasses.dataclass
class Params:
    """Numeric parameters of a planning workload (the planner's inputs)."""

    m: int = 100               # timesteps in the horizon
    n_coef: int = 11           # Bernstein coefficients per axis (degree 10)
    n_seg: int = 1             # set-point segments; p has 2*n_seg set-point entries
    inner_iters: int = 50      # K, projection iterations
    outer_iters: int = 5       # L, CEM iterations
    n_elite_c: int = 30        # ConstraintEliteSet size
    n_elite: int = 10          # EliteSet size q
    dt: float = 0.05
    rho: float = 1.0
    kp_lat: float = 1.0
    kv_lat: float = 2.0
    kp_lon: float = 1.0
    gamma: float = 0.9
    eta: float = 0.9
    cov_eps: float = 1e-6
    v_min: float = 0.1
    v_max: float = 25.0
    a_max: float = 6.0
    kappa_max: float = 0.2
    c_max: float = 4.0
    lane_margin: float = 1.0
    v_des_lo: float = 5.0      # first-iteration uniform range of v_d
    v_des_hi: float = 25.0
    goal: bool = False         # p also carries the goal positions x_f, y_f

    @property
    def d_p(self) -> int:
        return 2 * self.n_seg + (2 if self.goal else 0)


def make_scene(seed: int, n_lanes: int, n_obs: int, lane_width: float = 3.5,
               ego_vx=(10.0, 20.0), obs_x=(10.0, 80.0), obs_vx=(5.0, 15.0),
               obs_y_std: float = 0.2, axes=(2.8, 1.5), ego_lane: int | None = None,
               kappa_road: float = 0.0) -> Scene:
    """Dense-traffic scene: ego at x=0 on a lane centre, obstacles on lanes."""
    s = Stream(seed)
    centres = (np.arange(n_lanes) + 0.5) * lane_width
    lane = int(s.integers(0, n_lanes - 1, 1)[0]) if ego_lane is None else ego_lane
    ego = np.array([0.0, centres[lane], float(s.uniform(*ego_vx, 1)[0]), 0.0, 0.0, 0.0])
    obs = np.zeros((n_obs, 6))
    if n_obs:
        obs[:, 0] = s.uniform(*obs_x, n_obs)
        obs[:, 1] = centres[s.integers(0, n_lanes - 1, n_obs)] + s.normal(0.0, obs_y_std, n_obs)
        obs[:, 2] = s.uniform(*obs_vx, n_obs)
        obs[:, 4] = axes[0]
        obs[:, 5] = axes[1]
    return Scene(ego=ego, n_lanes=n_lanes, lane_width=lane_width,
                 kappa_road=kappa_road, obstacles=obs)


def curved_road(n_lanes: int, lane_width: float = 3.5, kappa: float = 0.01,
                bend=(40.0, 140.0), narrow_at: float | None = 90.0) -> np.ndarray:
    """Knots (s, kappa, lb, ub) of a road that enters a bend of curvature
    `kappa` over the arc-length interval `bend` (ramps of 20 m), and, from
    `narrow_at` on, loses its top lane (ramp of 10 m)."""
    w = n_lanes * lane_width
    s0, s1 = bend
    knots = [(0.0, 0.0), (s0, 0.0), (s0 + 20.0, kappa), (s1 - 20.0, kappa), (s1, 0.0)]
    ss = sorted({k[0] for k in knots} | ({narrow_at, narrow_at + 10.0} if narrow_at else set()))
    ks, kv = zip(*knots)
    rows = []
    for x in ss:
        ub = w if narrow_at is None else float(np.interp(x, [narrow_at, narrow_at + 10.0],
                                                         [w, w - lane_width]))
        rows.append((x, float(np.interp(x, ks, kv)), 0.0, ub))
    return np.array(rows)


def make_samples(seed: int, scene: Scene, B: int, n_seg: int,
                 v_range=(5.0, 25.0), goal_tf: float | None = None) -> np.ndarray:
    """B behavioural inputs p = [y_d,1..n_seg, v_d,1..n_seg] (Eq. behaviour_param):
    lateral set-points on lane centres, velocity set-points uniform.  With
    goal_tf (the horizon t_f in seconds) two goal entries follow: x_f = ego x +
    v t_f with v uniform in v_range, and y_f on a lane centre."""
    s = Stream(seed)
    centres = scene.lane_centres()
    p = np.empty((B, 2 * n_seg + (2 if goal_tf is not None else 0)))
    p[:, :n_seg] = centres[s.integers(0, scene.n_lanes - 1, B * n_seg)].reshape(B, n_seg)
    p[:, n_seg:2 * n_seg] = s.uniform(*v_range, B * n_seg).reshape(B, n_seg)
    if goal_tf is not None:
        p[:, 2 * n_seg] = float(scene.ego[0]) + goal_tf * s.uniform(*v_range, B)
        p[:, 2 * n_seg + 1] = centres[s.integers(0, scene.n_lanes - 1, B)]
    return p


# Workload recipes.  Sizes follow the five benchmark configurations of the
# planner: a small plain-FP64 case, the paper's dense-traffic sizes (n=1000
# samples, elites 150/50, Sec. V-A), batched scenes, served MPC episodes and
# a scale sweep.

def workload(index: int, scene_index: int = 0, **overrides):
    """Return (Params, Scene, B) for workload `index` (0, 1 or 4) and one scene."""
    seed = index * 1000 + scene_index
    if index == 0:
        prm = Params(m=100, n_coef=11, inner_iters=50, outer_iters=5, n_elite_c=30, n_elite=10)
        sc = make_scene(seed, n_lanes=2, n_obs=4, ego_lane=0)
        B = 64
    elif index == 1:
        prm = Params(m=100, n_coef=11, inner_iters=100, outer_iters=5, n_elite_c=150, n_elite=50)
        sc = make_scene(seed, n_lanes=4, n_obs=12)
        B = 1000
    elif index == 4:
        prm = Params(m=200, n_coef=16, inner_iters=100, outer_iters=5, n_elite_c=150, n_elite=50)
        sc = make_scene(seed, n_lanes=6, n_obs=30, obs_x=(10.0, 160.0))
        B = overrides.pop("B", 1024)
    else:
        raise ValueError("workload index must be 0, 1 or 4 (2 and 3 are multi-scene)")
    for k, v in overrides.items():
        setattr(prm, k, v)
    return prm, sc, B


def batched_workload(S: int = 256, seed: int = 2000, B_range=(256, 2048),
                     N_range=(4, 20), **overrides):
    """Workload of many scenes planned together: N ~ U{4..20}, B ~ U{256..2048}."""
    s = Stream(seed)
    Ns = s.integers(N_range[0], N_range[1], S)
    Bs = s.integers(B_range[0], B_range[1], S)
    scenes = [make_scene(seed + 1 + i, n_lanes=4, n_obs=int(Ns[i])) for i in range(S)]
    prm = Params(m=100, n_coef=11, inner_iters=100, outer_iters=5, n_elite_c=150, n_elite=50)
    for k, v in overrides.items():
        setattr(prm, k, v)
    return prm, scenes, [int(b) for b in Bs]

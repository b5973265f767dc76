"""Torch-facing convenience layer over the C ABI.

PyTorch supplies device memory and the current stream; every computation runs
in the CUDA library (binding.py marshals the arguments).
"""
from __future__ import annotations

import torch

from . import binding as B


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


def _need(t: torch.Tensor, shape, name: str):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Planner:
    """One planner context on the current CUDA device.

    params: object with the planner parameters (see scenegen.Params);
    prec: "fp32" (fused kernel), "fp64" (plain reference path), or a
          tensor-core mode "tf32", "bf16", "tf32x3" (contractions on tcgen05).
    """

    def __init__(self, params, prec: str = "fp32", max_obs: int = 32, max_samples: int = 4096,
                 max_scenes: int = 1):
        if not torch.cuda.is_available():
            raise RuntimeError("the planner runs on a CUDA GPU; none is available")
        self.prm = params
        self.prec = B.PRECISIONS[prec]
        self.cfg = B.make_config(params, self.prec, max_obs, max_samples, max_scenes)
        self.ctx = B.plan_init(self.cfg)
        self.n = params.n_coef
        self.d_p = 2 * params.n_seg + (2 if getattr(params, "goal", False) else 0)

    def close(self):
        if self.ctx is not None:
            B.plan_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- lower level
    def solve(self, scene, p: torch.Tensor, stream=None, want_xi: bool = True,
              want_status: bool = False):
        """(xi, r, c_u) of plan_solve, and the per-sample status (int32, PLAN_OK or
        PLAN_ENONFINITE) as a fourth entry when want_status."""
        Bn = p.shape[0]
        _need(p, (Bn, self.d_p), "p")
        dev = p.device
        xi = torch.empty((Bn, 2 * self.n), dtype=torch.float64, device=dev) if want_xi else None
        r = torch.empty(Bn, dtype=torch.float64, device=dev)
        cu = torch.empty(Bn, dtype=torch.float64, device=dev)
        st = torch.empty(Bn, dtype=torch.int32, device=dev) if want_status else None
        B.plan_solve(self.ctx, scene, _ptr(p), Bn, _ptr(xi), _ptr(r), _ptr(cu), _ptr(st) or None,
                     _stream(stream))
        return (xi, r, cu, st) if want_status else (xi, r, cu)

    def solve_batch(self, scenes, Bs, p: torch.Tensor, stream=None, want_status: bool = False):
        tot = int(sum(Bs))
        _need(p, (tot, self.d_p), "p")
        xi = torch.empty((tot, 2 * self.n), dtype=torch.float64, device=p.device)
        r = torch.empty(tot, dtype=torch.float64, device=p.device)
        cu = torch.empty(tot, dtype=torch.float64, device=p.device)
        st = torch.empty(tot, dtype=torch.int32, device=p.device) if want_status else None
        B.plan_solve_batch(self.ctx, scenes, Bs, _ptr(p), _ptr(xi), _ptr(r), _ptr(cu),
                           _ptr(st) or None, _stream(stream))
        return (xi, r, cu, st) if want_status else (xi, r, cu)

    # -------------------------------------------------------------- Alg. 1
    def upload(self, scenes, stream=None):
        B.plan_upload_scenes(self.ctx, scenes, _stream(stream))

    def set_state(self, slot: int, mu=None, sigma=None, seed: int = 0, step: int = 0, fresh=None,
                  stream=None):
        B.plan_set_state(self.ctx, slot, B.make_state(self.d_p, mu, sigma, seed, step, fresh),
                         _stream(stream))

    def get_state(self, slot: int, stream=None):
        st = B.plan_get_state(self.ctx, slot, _stream(stream))
        mu, sigma = B.state_arrays(st, self.d_p)
        return dict(mu=mu, sigma=sigma, seed=st.seed, step=st.episode_step, fresh=st.fresh)

    def step_resident(self, Bs, stream=None):
        B.plan_step_resident(self.ctx, Bs, _stream(stream))

    def get_result(self, slot: int, stream=None):
        r = B.plan_get_result(self.ctx, slot, _stream(stream))
        return dict(p=list(r.p[:self.d_p]), xi=list(r.xi[:2 * self.n]), cost=r.cost,
                    resid=r.resid, cu=r.cu, index=r.index)

    def step(self, scene, Bn: int, mu=None, sigma=None, seed: int = 0, step: int = 0, stream=None):
        st = B.make_state(self.d_p, mu, sigma, seed, step)
        r = B.plan_step(self.ctx, scene, st, Bn, _stream(stream))
        mu1, sg1 = B.state_arrays(st, self.d_p)
        return dict(p=list(r.p[:self.d_p]), xi=list(r.xi[:2 * self.n]), cost=r.cost, resid=r.resid,
                    cu=r.cu, index=r.index, mu=mu1, sigma=sg1, step=st.episode_step)

    # -------------------------------------------------------------- tuning
    def set_tuning(self, warps_per_sample: int, samples_per_cta: int):
        B.plan_set_tuning(self.ctx, warps_per_sample, samples_per_cta)

    def set_persistent(self, mode):
        """Launch form of the fused FP32 kernel: "auto", "off" or "on"."""
        B.plan_set_persistent(self.ctx, mode)

    def autotune(self, scene, Bn: int, stream=None):
        return B.plan_autotune(self.ctx, scene, Bn, _stream(stream))

    # -------------------------------------------------------------- single stages
    def select_elites(self, r: torch.Tensor, cu: torch.Tensor, n_c: int, q: int, stream=None):
        Bn = r.shape[0]
        _need(r, (Bn,), "r")
        _need(cu, (Bn,), "cu")
        elite = torch.empty(q, dtype=torch.int32, device=r.device)
        B.plan_select_elites(self.ctx, _ptr(r), _ptr(cu), Bn, n_c, q, _ptr(elite), _stream(stream))
        return elite

    def update_distribution(self, p_elite: torch.Tensor, cost: torch.Tensor, mu: torch.Tensor,
                            sigma: torch.Tensor, stream=None):
        q = p_elite.shape[0]
        _need(p_elite, (q, self.d_p), "p_elite")
        _need(cost, (q,), "cost")
        _need(mu, (self.d_p,), "mu")
        _need(sigma, (self.d_p, self.d_p), "sigma")
        B.plan_update_distribution(self.ctx, _ptr(p_elite), _ptr(cost), q, _ptr(mu), _ptr(sigma),
                                   _stream(stream))

    # -------------------------------------------------------------- Step-1 layer
    def qp_forward(self, p: torch.Tensor, b0: torch.Tensor, stream=None):
        """xi (B, 2n) of the Step-1 QP for each row of p (B, d_p) and b0 (B, 6)."""
        Bn = p.shape[0]
        _need(p, (Bn, self.d_p), "p")
        _need(b0, (Bn, 6), "b0")
        xi = torch.empty((Bn, 2 * self.n), dtype=torch.float64, device=p.device)
        B.plan_qp_forward(self.ctx, _ptr(p), _ptr(b0), Bn, _ptr(xi), _stream(stream))
        return xi

    def qp_backward(self, g: torch.Tensor, want_b0: bool = True, stream=None):
        """(dL/dp, dL/db0) for g = dL/dxi (B, 2n); dL/db0 is None unless wanted."""
        Bn = g.shape[0]
        _need(g, (Bn, 2 * self.n), "g")
        gp = torch.empty((Bn, self.d_p), dtype=torch.float64, device=g.device)
        gb = torch.empty((Bn, 6), dtype=torch.float64, device=g.device) if want_b0 else None
        B.plan_qp_backward(self.ctx, _ptr(g), Bn, _ptr(gp), _ptr(gb), _stream(stream))
        return gp, gb

    def qp_layer(self, p: torch.Tensor, b0: torch.Tensor):
        """The Step-1 layer as a torch.autograd function of (p, b0)."""
        return _QPLayer.apply(p, b0, self)

    def sample(self, scene, Bn: int, l: int, seed: int, step: int = 0, mu=None, sigma=None,
               stream=None, device=None):
        p = torch.empty((Bn, self.d_p), dtype=torch.float64, device=device or "cuda")
        B.plan_sample(self.ctx, scene, mu, sigma, int(mu is None), l, seed, step, Bn, _ptr(p),
                      _stream(stream))
        return p


class _QPLayer(torch.autograd.Function):
    """Forward and backward through the library's Step-1 layer kernels."""

    @staticmethod
    def forward(ctx, p, b0, planner):
        ctx.planner = planner
        return planner.qp_forward(p.contiguous(), b0.contiguous())

    @staticmethod
    def backward(ctx, g):
        gp, gb = ctx.planner.qp_backward(g.contiguous(), want_b0=ctx.needs_input_grad[1])
        return gp, gb, None


class Server:
    """Continuous-batching serving loop over the C ABI (plan_server_*).

    Each request is one MPC cycle of an episode; episodes keep their sampling
    distribution on the device between cycles."""

    def __init__(self, params, prec: str = "fp32", max_obs: int = 32, max_samples: int = 8192,
                 max_scenes: int = 32, max_executors: int = 4, device_budget: int = 4 << 30,
                 max_episodes: int = 1024):
        p = B.PRECISIONS[prec]
        self.cfg = B.make_config(params, p, max_obs, max_samples, max_scenes)
        self.srv = B.plan_server_create(self.cfg, max_executors, device_budget, max_episodes)
        self.n = params.n_coef
        self.d_p = 2 * params.n_seg + (2 if getattr(params, "goal", False) else 0)

    def submit(self, scene, Bn: int, m: int = 0, episode: int = 0, seed: int = 0, fresh: int = 0):
        return B.plan_submit(self.srv, scene, Bn, m, episode, seed, fresh)

    def poll(self, ticket: int, timeout_us: int = 1_000_000):
        st, r, lat = B.plan_poll(self.srv, ticket, timeout_us)
        if st == B.PLAN_ETIMEOUT:
            return None
        return dict(p=list(r.p[:self.d_p]), xi=list(r.xi[:2 * self.n]), cost=r.cost,
                    resid=r.resid, cu=r.cu, index=r.index, latency_us=lat)

    def poll_any(self, timeout_us: int = 0):
        """(ticket, result) of the first completed request, or None after
        timeout_us without a completion."""
        st, t, r, lat = B.plan_poll_any(self.srv, timeout_us)
        if st == B.PLAN_ETIMEOUT:
            return None
        return t, dict(p=list(r.p[:self.d_p]), xi=list(r.xi[:2 * self.n]), cost=r.cost,
                       resid=r.resid, cu=r.cu, index=r.index, latency_us=lat)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        import time
        t_end = time.time() + timeout_s
        while time.time() < t_end:
            r = self.poll(ticket, 100_000)
            if r is not None:
                return r
        raise TimeoutError(f"ticket {ticket} not done in {timeout_s} s")

    def end_episode(self, episode: int):
        B.plan_end_episode(self.srv, episode)

    def info(self):
        return B.plan_server_info(self.srv)

    def close(self):
        if self.srv is not None:
            B.plan_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def advance(params, scene, xi, steps: int = 5):
    """Next MPC scene after executing `steps` elements of plan xi (plan_advance)."""
    cfg = B.make_config(params, B.PLAN_PREC_FP32, 0, 1)
    return B.plan_advance(cfg, scene, xi, steps)

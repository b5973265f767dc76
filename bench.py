#!/usr/bin/env python3
"""Benchmark of the GB300 bi-level planner on the dense-traffic workload.

One step = one MPC cycle = Alg. 1 with L = 5 outer iterations over one scene
(4 lanes, 12 constant-velocity obstacles), B = 1000 sampled behavioural inputs,
m = 100 timesteps, 11 Bernstein coefficients per axis, K = 100 projection
iterations, ConstraintEliteSet 150 and EliteSet 50 (the paper's sizes).

value  : sample-iterations / s = B * K * L / device time of one cycle, inputs
         resident in HBM, CUDA events on the launching stream, L2 flushed
         (256 MiB write) before every timed cycle.  Every cycle is a planning
         call of its own (its first outer iteration samples the behavioural
         prior, Alg. 1 line 2), so no cycle inherits a distribution that has
         already converged on one trajectory.
e2e    : the same metric through plan_step with host buffers (scene and
         distribution go up, best pair and distribution come back), the same
         sequence of planning calls.
plain_fp64 : the same cycle on the plain float64 path (reference GPU path).
roofline   : the fused solve kernel against the FP32 FMA pipe.
latency_ms : p50 / p99 over --latency-cycles cycles after 50 warm-up cycles,
             on the device (graph) and through plan_step (host wall clock).
cpu_baseline: the FP64 oracle on a bounded sample, one host thread;
cpu_baseline_all_cores: the same with one process per host core.
scale_point : the scale sweep's largest point (6 lanes, 30 obstacles, m = 200,
              n = 16, B = 32 768): ms per cycle, value and the fused solve's
              fraction of the FP32 pipe, with its own clock record.
batched     : the 256-scene workload (N ~ U{4..20}, B ~ U{256..2048}): ms per
              graph-captured step, value, solve fraction, clocks.
serving     : the served MPC loop (Poisson arrivals over 64 episodes) at 600 and
              1000 requests/s, 3 s of arrivals each: latency from arrival to
              completion, throughput, drops.
precision   : one B = 1000 solve per arithmetic mode against the plain FP64 GPU
              path, and the same with goal entries in p.

--impl reference times the FP64 CPU oracle on the same metric instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("dense-traffic single scene: 4 lanes, 12 obstacles, B=1000 samples, m=100 steps, "
            "n=11 coefficients/axis, K=100 projection iterations, L=5 CEM iterations, elites 150/50")
METRIC = "plan solves/sec (samples x inner iters x outer iters)"
UNIT = "sample-iters/s"
FP32_LANES_PER_SM = 128
SM_COUNT_NOMINAL = 152
# DRAM bytes (read + write) of one fused solve of this workload, by kernel shape
# (warps per sample, samples per CTA), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum; summary and command under profiles/), together with the
# SHA-256 of the kernel source it was taken on.  bench.py reports the figure only
# while the source still has that hash; otherwise traffic is null.
FUSED_TRAFFIC = {
    "source_sha256": "61d70982cf964012b25ce8b67939f313e572e59f2d52be44a5c69d7a6b681d5d",
    "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum of the third solve of "
               "python -m paper_2212_02224_gb300.profile_solve --prec fp32 --shape W S --reps 3 "
               "(summary and command under profiles/)",
    "bytes": {(1, 1): 107008, (1, 2): 98048, (1, 4): 94208, (1, 5): 92672, (1, 6): 92416,
              (1, 7): 92928, (1, 8): 91904, (2, 1): 97536, (2, 2): 89344, (2, 4): 85760,
              (4, 1): 112640},
}
FUSED_KERNEL_SOURCES = ("paper_2212_02224_gb300/csrc/fused_kernel.cuh",
                        "paper_2212_02224_gb300/csrc/k_fused.cu")


def fused_source_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in FUSED_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def fused_traffic(shape):
    """(bytes per launch or None, note) for the fused kernel of this shape."""
    if FUSED_TRAFFIC["source_sha256"] != fused_source_sha256():
        return None, "no ncu capture of the current kernel source"
    b = FUSED_TRAFFIC["bytes"].get(tuple(shape))
    return b, (FUSED_TRAFFIC["capture"] if b is not None else "shape not captured")


def algorithmic_flops_per_sample_iter(m, n, N, n_eq=3):
    """Per sample and Alg. 2 iteration: forward and transposed contractions
    (24 m n), obstacle projection (12 N m), velocity / acceleration / lane rows
    (40 m), multiplier and xi-step updates (4 n^2 + 4 n n_eq)."""
    return 24 * m * n + 12 * N * m + 40 * m + 4 * n * n + 4 * n * n_eq


# ----------------------------------------------------------------------------- CPU oracle

_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg
prm, sc, B = sg.workload(1)
basis = bernstein(prm.m, prm.n_coef, prm.dt)
p = sg.make_samples({seed}, sc, {nsamp}, prm.n_seg)
lower.solve(p[:2], sc, prm, basis, iters=2)          # warm caches / imports
t0 = time.perf_counter(); reps = 0
while True:
    lower.solve(p, sc, prm, basis)
    reps += 1
    if time.perf_counter() - t0 >= {budget}:
        break
dt = time.perf_counter() - t0
print(json.dumps(dict(units=reps * {nsamp} * prm.inner_iters, seconds=dt, reps=reps)))
"""


_ONE_THREAD = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def run_oracle(nsamp=40, budget=12.0):
    env = dict(os.environ, **_ONE_THREAD)
    code = _ORACLE_SNIPPET.format(root=ROOT, nsamp=nsamp, budget=budget, seed=303)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    return dict(value=res["units"] / res["seconds"], unit=UNIT, cores=1, kind="oracle",
                sample=f"{res['reps']} x lower-level solve of {nsamp} samples of the workload "
                       f"(K=100), numpy float64, one thread; one sample-iteration = one Alg. 2 "
                       f"iteration of one sample")


def run_oracle_all_cores(nsamp=20, budget=12.0):
    """The same oracle solve in one single-threaded process per host core, each
    on its own samples, all started together: the samples split across the
    cores with no shared state.  value = all processes' sample-iterations over
    the longest process's time."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    env = dict(os.environ, **_ONE_THREAD)
    procs = [subprocess.Popen([sys.executable, "-c", _ORACLE_SNIPPET.format(
                 root=ROOT, nsamp=nsamp, budget=budget, seed=1000 + i)],
                 stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for i in range(cores)]
    res = []
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        if pr.returncode != 0:
            raise RuntimeError(err)
        res.append(json.loads(out.strip().splitlines()[-1]))
    units = sum(r["units"] for r in res)
    secs = max(r["seconds"] for r in res)
    return dict(value=units / secs, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{cores} processes x (>= {min(r['reps'] for r in res)} lower-level solves "
                       f"of {nsamp} samples of the workload, K=100), numpy float64, one thread "
                       f"each, samples split across processes")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return dict(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                    reasons=reasons, samples=len(rows))


def clocks_rejected(clocks) -> bool:
    """True when a timed region's clock record rejects it: a hardware or thermal
    slowdown was active, or the SM clock sat below 90 % of its maximum with no
    reason given (a clock held by an earlier user).  sw_power_cap alone is kept."""
    if not clocks:
        return False
    if set(clocks["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    return not clocks["reasons"] and clocks["sm_mhz"] < 0.9 * clocks["sm_max_mhz"]


# ----------------------------------------------------------------------------- replicas

class Ranks:
    """One process per GPU (torchrun environment): rank, world size, barrier and
    the max-over-ranks reduction of a timing.  Replicas run independent scenes,
    so the only collectives are this barrier and this reduction."""

    def __init__(self, backend="nccl", device="cuda"):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if device == "cuda":
            torch.cuda.set_device(self.local)
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", self.local)} if device == "cuda" else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64,
                         device=self.device if self.device == "cpu" else f"cuda:{self.local}")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def replica_value(units_per_step: float, steps: int, slowest_s: float, world: int) -> float:
    """Whole-job throughput: every replica processes units_per_step per step;
    the job takes as long as its slowest rank."""
    return world * units_per_step * steps / slowest_s


# ----------------------------------------------------------------------------- GPU arm

def precision_modes(prm, sc, p, flush, stream, reps=10):
    """Solve time of each arithmetic mode on the same samples (CUDA events, L2
    flushed) and the error of its results against the plain FP64 GPU path:
    largest trajectory-position difference (m), residual difference and
    relative cost difference over all samples."""
    import numpy as np
    import torch

    from paper_2212_02224_gb300.planner import Planner

    B = p.shape[0]
    n, m = prm.n_coef, prm.m
    # Bernstein rows W[t][k] of the positions, in float64 on the host
    from math import comb
    tau = np.arange(m) / (m - 1)
    W = np.stack([comb(n - 1, k) * tau ** k * (1 - tau) ** (n - 1 - k) for k in range(n)], axis=1)

    def solve(prec):
        pl = Planner(prm, prec=prec, max_obs=16, max_samples=B)
        for _ in range(3):
            pl.solve(sc, p, want_xi=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            pl.solve(sc, p, want_xi=False)
            b.record(stream)
        xi, r, cu = pl.solve(sc, p)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
        pl.close()
        return ms, out

    def pos_err(xi, ref_xi):
        return float(np.hypot((xi[:, :n] - ref_xi[:, :n]) @ W.T, (xi[:, n:] - ref_xi[:, n:]) @ W.T).max())

    ms64, ref = solve("fp64")
    res = {"reference": "plain FP64 GPU path (itself within 1e-6 of the FP64 oracle)",
           "errors": "largest over the samples: Euclidean distance between the two plans' "
                     "points at any t, |r - r_ref|, |c_u - c_u,ref| / |c_u,ref|",
           "fp64": {"solve_ms": ms64}}
    for prec in ("fp32", "tf32x3", "tf32", "bf16"):
        ms, (xi, r, cu) = solve(prec)
        pos = pos_err(xi, ref[0])
        res[prec] = {"solve_ms": ms, "max_pos_err_m": float(pos),
                     "max_resid_err": float(np.abs(r - ref[1]).max()),
                     "max_cost_rel_err": float((np.abs(cu - ref[2]) /
                                                np.maximum(1e-12, np.abs(ref[2]))).max()),
                     "contractions": "CUDA-core FP32 FMA" if prec == "fp32" else
                                     f"tcgen05 kind::{'f16 (bf16)' if prec == 'bf16' else 'tf32'}"
                                     f"{' x3 split' if prec == 'tf32x3' else ''}, FP32 accumulate"}
    # goal entries of p (Eq. behaviour_param's x_f, y_f; Eq. final_boundary rows):
    # the same scene and set-points with goals drawn as the first-iteration prior
    import copy
    from paper_2212_02224_gb300 import scenegen as sg
    gprm = copy.copy(prm)
    gprm.goal = True
    pg = torch.tensor(sg.make_samples(303, sc, B, prm.n_seg, goal_tf=(prm.m - 1) * prm.dt),
                      dtype=torch.float64, device="cuda")
    goal = {}
    outs = {}
    for prec in ("fp64", "fp32"):
        pl = Planner(gprm, prec=prec, max_obs=16, max_samples=B)
        for _ in range(3):
            pl.solve(sc, pg, want_xi=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            pl.solve(sc, pg, want_xi=False)
            b.record(stream)
        xi, r, cu = pl.solve(sc, pg)
        torch.cuda.synchronize()
        outs[prec] = (xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy())
        goal[prec] = {"solve_ms": statistics.median(a.elapsed_time(b) for a, b in ev)}
        pl.close()
    xi, r, cu = outs["fp32"]
    xr, rr, cr = outs["fp64"]
    e = np.hypot((xi[:, :n] - xr[:, :n]) @ W.T, (xi[:, n:] - xr[:, n:]) @ W.T).max(axis=1)
    goal["fp32"].update({
        "max_pos_err_m": float(e.max()), "median_pos_err_m": float(np.median(e)),
        "samples_over_1e-3_m": int((e > 1e-3).sum()),
        "max_cost_rel_err": float((np.abs(cu - cr) / np.maximum(1e-12, np.abs(cr))).max())})
    goal["config"] = ("p = [y_d, v_d, x_f, y_f] (d_p = 4), x_f = x0 + U[5, 25] t_f, y_f a lane "
                      "centre; terminal rows x(t_f), y(t_f), ydot(t_f) in A_eq; errors against "
                      "the plain FP64 GPU path; samples over 1e-3 m are the ill-conditioned "
                      "ones (hard braking to the goal)")
    res["goal"] = goal
    return res


def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Planner

    ranks = Ranks("nccl", "cuda")
    world, rank, local = ranks.world, ranks.rank, ranks.local
    barrier = ranks.barrier

    prm, sc, B = sg.workload(1)
    K, L = prm.inner_iters, prm.outer_iters
    units = B * K * L
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # ---- value: resident inputs, graph-captured cycle
    pl = Planner(prm, prec="fp32", max_obs=16, max_samples=B)
    shape = pl.autotune(sc, B)          # fused-kernel shape for this workload (setup, untimed)
    pl.upload([sc])

    def fresh(i):
        # every cycle is a planning call of its own: its first outer iteration
        # samples the behavioural prior (Alg. 1 line 2); the state upload is
        # queued before the timed region starts
        pl.set_state(0, seed=1234 + rank, step=i)

    for i in range(args.warmup):
        fresh(i)
        pl.step_resident([B])
    barrier()

    def measure():
        # the timed cycles, then the latency run; the clock sampler covers both
        # so that its 200 ms samples fall inside device-timed work
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            barrier()
            for i in range(args.steps):
                flush.zero_()
                fresh(args.warmup + i)
                starts[i].record(stream)
                pl.step_resident([B])
                ends[i].record(stream)
            barrier()
            # ---- latency: per-cycle device time over many cycles after 50 warm-up cycles
            lat = []
            if args.latency_cycles > 0:
                for i in range(50):
                    fresh(i)
                    pl.step_resident([B])
                lat = _timed(lambda: pl.step_resident([B]), args.latency_cycles, flush, stream,
                             prep=fresh)
        return [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)], lat, clk.summary()

    step_ms, lat_ms, clocks = measure()
    bad = clocks_rejected(clocks)
    remeasured = False
    if ranks.max(1.0 if bad else 0.0) > 0.5:      # decided together: measure() has barriers
        # a slowdown, or clocks held below their maximum with no reason: measure once more
        step_ms, lat_ms, clocks = measure()
        remeasured = True
    if clocks is not None:
        clocks["remeasured"] = remeasured
    total_s = ranks.max(sum(step_ms) / 1e3)
    value = replica_value(units, args.steps, total_s, world)

    # ---- e2e: through host buffers (plan_step), wall clock per cycle
    e2e_ms = []
    n_e2e = max(args.steps, args.latency_cycles)
    for i in range(max(args.warmup, 50 if args.latency_cycles > 0 else 0) + n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl.step(sc, B, seed=1234 + rank, step=i)      # a fresh planning call, as above
        dt_ms = (time.perf_counter() - t0) * 1e3
        if i >= max(args.warmup, 50 if args.latency_cycles > 0 else 0):
            e2e_ms.append(dt_ms)
    e2e_total = ranks.max(sum(e2e_ms) / 1e3)
    e2e_value = replica_value(units, len(e2e_ms), e2e_total, world)
    # plan_step moves, per cycle, from pinned host memory to the device: the
    # scene record, its obstacles (48 B each) and the sampling state; back: the
    # final state with the best pair and the timeout flag (8 B).  Record sizes:
    # scene 10 doubles + 4 ints + 8 road knots x 4 doubles; sampling state
    # mu, best p (PLAN_MAX_DP each), sigma and its Cholesky factor (PLAN_MAX_DP^2
    # each), best xi (32), 3 doubles, 2 uint64, 4 ints
    from paper_2212_02224_gb300.binding import PLAN_MAX_DP as DPM
    dev_scene = 8 * 10 + 4 * 4 + 8 * 32
    dev_cem = 8 * (2 * DPM + 2 * DPM * DPM + 32 + 3) + 16 + 16
    h2d = dev_scene + 48 * sc.n_obs + dev_cem
    d2h = dev_cem + 8

    # ---- roofline of the fused solve kernel (timed alone on this stream)
    p = torch.tensor(sg.make_samples(303, sc, B, prm.n_seg), dtype=torch.float64, device="cuda")
    for _ in range(3):
        pl.solve(sc, p, want_xi=False)
    reps = 20
    ks = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for i in range(reps):
        flush.zero_()
        ks[i].record(stream)
        pl.solve(sc, p, want_xi=False)
        ke[i].record(stream)
    torch.cuda.synchronize()
    kern_ms = statistics.mean(s.elapsed_time(e) for s, e in zip(ks, ke))
    flops = algorithmic_flops_per_sample_iter(prm.m, prm.n_coef, sc.n_obs) * B * K
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_clock = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * 2 * peak_clock * 1e6 / 1e12
    achieved = flops / (kern_ms * 1e-3) / 1e12
    pl.close()
    traffic_b, traffic_note = fused_traffic(shape)
    from paper_2212_02224_gb300 import binding
    probe = binding.plan_probe_alu()

    # ---- the scale sweep's largest point (B = 32 768) and the 256-scene batched
    # step, so that the default line reports them too (each with its own clocks)
    extra = {}
    if not args.skip_extra:
        extra["scale_point"] = scale_point(32768, max(3, min(args.steps, 5)), args.warmup, flush,
                                           stream, sms, local)
        extra["batched"] = batched_point(max(3, min(args.steps, 5)), args.warmup, flush, stream,
                                         sms, local)
        # the served MPC loop below and at its saturation rate, 3 s of arrivals each
        extra["serving"] = []
        for rate in (600.0, 1000.0):
            sv = serve(rate, 3.0)
            extra["serving"].append({
                "rate_req_s": rate, "achieved_req_s": sv["achieved_req_s"], "value": sv["value"],
                "unit": UNIT, "p50_ms": sv["latency_ms"]["p50"], "p99_ms": sv["latency_ms"]["p99"],
                "server_p50_ms": sv["server_latency_ms"]["p50"],
                "server_p99_ms": sv["server_latency_ms"]["p99"], "completed": sv["completed"],
                "dropped": sv["dropped"], "config": sv["config"]["workload"]})

    # ---- precision modes: one lower-level solve of the same B = 1000 samples per
    # mode, timed alone, and its error against the plain FP64 GPU path
    precision = precision_modes(prm, sc, p, flush, stream) if not args.skip_fp64 else None

    # ---- plain FP64 path, same cycle
    plain = None
    if not args.skip_fp64:
        pf = Planner(prm, prec="fp64", max_obs=16, max_samples=B)
        pf.upload([sc])
        pf.set_state(0, seed=1234 + rank)
        pf.step_resident([B])
        torch.cuda.synchronize()
        n64 = max(1, min(args.steps, 3))
        fs = [torch.cuda.Event(enable_timing=True) for _ in range(n64)]
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(n64)]
        for i in range(n64):
            flush.zero_()
            pf.set_state(0, seed=1234 + rank, step=i)
            fs[i].record(stream)
            pf.step_resident([B])
            fe[i].record(stream)
        torch.cuda.synchronize()
        ms64 = statistics.mean(s.elapsed_time(e) for s, e in zip(fs, fe))
        plain = dict(value=units / (ms64 * 1e-3), unit=UNIT, ms_per_step=ms64, steps=n64)
        pf.close()

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = run_oracle()
        cpu_all = run_oracle_all_cores()

    if rank == 0:
        lat = lat_ms or step_ms
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas{world}",
                       "l2": "flushed before every timed step (256 MiB write)",
                       "graph": "whole cycle captured as one CUDA graph",
                       "cycle": "each timed cycle is a fresh planning call (first outer "
                                "iteration samples the behavioural prior)",
                       "fused_shape": {"warps_per_sample": shape[0], "samples_per_cta": shape[1]}},
            "latency_ms": {"p50": statistics.median(lat),
                           "p99": float(np.percentile(lat, 99)),
                           "cycles": len(lat),
                           "e2e_p50": statistics.median(e2e_ms),
                           "e2e_p99": float(np.percentile(e2e_ms, 99)),
                           "e2e_cycles": len(e2e_ms),
                           "warmup_cycles": 50 if lat_ms else args.warmup,
                           "basis": "device time per graph-captured cycle (L2 flushed before "
                                    "each); e2e = wall time per plan_step call"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per cycle: sampling, solve and selection in each outer iteration, and
            # the normals of iterations 2..L on the graph's side branch
            "gpu_launches": args.steps * (3 * L + max(0, L - 1)),
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (value / plain["value"]) if plain else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": traffic_b,
                         "traffic_source": traffic_note,
                         "kernel": f"fused_kernel (n=11, {shape[0]} warp(s)/sample, "
                                   f"{shape[1]} sample(s)/CTA; one lower-level solve, B=1000, K=100)",
                         "kernel_ms": kern_ms,
                         "peak_basis": f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 flop x "
                                       f"{peak_clock:.0f} MHz",
                         "probe": {k: v for k, v in probe.items()},
                         "probe_basis": "plan_probe_alu: independent FFMA / FFMA2 / DFMA / "
                                        "MUFU rsqrt chains, 8 CTAs x 256 threads per SM"},
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "clocks": clocks,
            "precision": precision,
            **extra,
        }
        print(json.dumps(line))
    ranks.close()


# ----------------------------------------------------------------------------- reference arm

def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    per_step = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        r = run_oracle(nsamp=20, budget=per_step)
        if i >= args.warmup:
            vals.append(r)
    value = statistics.mean(v["value"] for v in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "none (CPU oracle)"},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                         "sample": vals[0]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- other workloads

def _timed(fn, reps, flush, stream, prep=None):
    """Device time of `reps` calls of fn, L2 flushed before each; prep(i) runs
    (and queues its work) before each timed region starts."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for i, (a, b) in enumerate(ev):
        flush.zero_()
        if prep is not None:
            prep(i)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def fp32_peak_tflops(sms, clocks):
    clk = (clocks or {}).get("sm_max_mhz") or 2070.0
    return sms * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12


def scale_point(B, steps, warmup, flush, stream, sms, index=0):
    """One point of the scale sweep (6 lanes, 30 obstacles, m = 200, n = 16,
    K = 100, L = 5): device time per graph-captured cycle (fresh planning calls,
    L2 flushed), and the fused solve timed alone against the FP32 pipe."""
    import torch
    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Planner
    prm, sc, _ = sg.workload(4, B=B)
    pl = Planner(prm, prec="fp32", max_obs=32, max_samples=B)
    shape = pl.autotune(sc, B)
    pl.upload([sc])

    def fresh(i):
        pl.set_state(0, seed=7, step=i)

    for i in range(warmup):
        fresh(i)
        pl.step_resident([B])
    p = torch.tensor(sg.make_samples(3, sc, B, prm.n_seg), device="cuda")
    with ClockSampler(index) as clk:
        ms = _timed(lambda: pl.step_resident([B]), steps, flush, stream, prep=fresh)
        ks = _timed(lambda: pl.solve(sc, p, want_xi=False), 5, flush, stream)
    clocks = clk.summary()
    pl.close()
    flops = algorithmic_flops_per_sample_iter(prm.m, prm.n_coef, sc.n_obs) * B * prm.inner_iters
    solve_ms = statistics.median(ks)
    tflops = flops / (solve_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(sms, clocks)
    return {"config": f"6 lanes, N=30, m=200, n=16, B={B}, K=100, L=5", "B": B,
            "fused_shape": {"warps_per_sample": shape[0], "samples_per_cta": shape[1]},
            "ms_per_cycle": statistics.median(ms), "cycles": len(ms),
            "value": B * prm.inner_iters * prm.outer_iters / (statistics.median(ms) / 1e3),
            "unit": UNIT, "solve_ms": solve_ms, "solve_tflops": tflops, "peak_tflops": peak,
            "frac": tflops / peak, "clocks": clocks}


def batched_point(steps, warmup, flush, stream, sms, index=0):
    """The batched workload (256 scenes, N ~ U{4..20}, B ~ U{256..2048}): one
    graph-captured Alg. 1 run over all scenes per step, and its fused solve
    timed alone against the FP32 pipe."""
    import torch
    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Planner
    prm, scenes, Bs = sg.batched_workload(S=256)
    tot = sum(Bs)
    pl = Planner(prm, prec="fp32", max_obs=20, max_samples=tot, max_scenes=len(scenes))
    pl.set_tuning(1, 2)
    pl.upload(scenes)

    def fresh(i):
        for k in range(len(scenes)):
            pl.set_state(k, seed=100 + k, step=i)

    for i in range(warmup):
        fresh(i)
        pl.step_resident(Bs)
    import numpy as np
    p = torch.tensor(np.concatenate([sg.make_samples(9 + i, scenes[i], Bs[i], prm.n_seg)
                                     for i in range(len(scenes))]), device="cuda")
    with ClockSampler(index) as clk:
        ms = _timed(lambda: pl.step_resident(Bs), steps, flush, stream, prep=fresh)
        ks = _timed(lambda: pl.solve_batch(scenes, Bs, p), 3, flush, stream)
    clocks = clk.summary()
    pl.close()
    flops = sum(algorithmic_flops_per_sample_iter(prm.m, prm.n_coef, sc.n_obs) * b * prm.inner_iters
                for sc, b in zip(scenes, Bs))
    solve_ms = statistics.median(ks)
    tflops = flops / (solve_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(sms, clocks)
    units = tot * prm.inner_iters * prm.outer_iters
    return {"config": "256 scenes, N~U{4..20}, B~U{256..2048} (total %d), m=100, n=11, K=100, "
                      "L=5, one CUDA graph per step" % tot,
            "ms_per_step": statistics.median(ms), "steps": len(ms),
            "value": units / (statistics.median(ms) / 1e3), "unit": UNIT,
            "scenes_per_s": len(scenes) / (statistics.median(ms) / 1e3),
            "solve_ms": solve_ms, "solve_tflops": tflops, "peak_tflops": peak,
            "frac": tflops / peak, "clocks": clocks}


def batched_arm(args):
    """Many scenes per MPC cycle: 256 scenes, N ~ U{4..20}, B ~ U{256..2048},
    one graph-captured Alg. 1 run over all of them per step."""
    import torch
    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Planner
    prm, scenes, Bs = sg.batched_workload(S=256)
    tot = sum(Bs)
    pl = Planner(prm, prec="fp32", max_obs=20, max_samples=tot, max_scenes=len(scenes))
    pl.set_tuning(1, 2)
    pl.upload(scenes)

    def fresh(i):      # every cycle a planning call of its own, as in the dense arm
        for k in range(len(scenes)):
            pl.set_state(k, seed=100 + k, step=i)

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        fresh(i)
        pl.step_resident(Bs)
    with ClockSampler(0) as clk:
        ms = _timed(lambda: pl.step_resident(Bs), args.steps, flush, stream, prep=fresh)
    units = tot * prm.inner_iters * prm.outer_iters
    print(json.dumps({
        "metric": METRIC, "workload": "batched", "value": units * len(ms) / (sum(ms) / 1e3),
        "unit": UNIT, "scenes_per_s": len(scenes) * len(ms) / (sum(ms) / 1e3),
        "ms_per_step": statistics.mean(ms), "p50_ms": statistics.median(ms),
        "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "256 scenes, N~U{4..20}, B~U{256..2048} (total %d), m=100, n=11, "
                               "K=100, L=5, one CUDA graph per step" % tot},
        "clocks": clk.summary()}))
    pl.close()


def scale_arm(args):
    """One scene, 6 lanes, 30 obstacles, m=200, n=16, B from 1k to 32k."""
    import torch
    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Planner
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for B in (1024, 2048, 4096, 8192, 16384, 32768):
        prm, sc, _ = sg.workload(4, B=B)
        pl = Planner(prm, prec="fp32", max_obs=32, max_samples=B)
        pl.autotune(sc, B)
        pl.upload([sc])

        def fresh(i, pl=pl):
            pl.set_state(0, seed=7, step=i)

        for i in range(args.warmup):
            fresh(i)
            pl.step_resident([B])
        ms = _timed(lambda: pl.step_resident([B]), max(3, args.steps // 4), flush, stream, prep=fresh)
        p = torch.tensor(sg.make_samples(3, sc, B, prm.n_seg), device="cuda")
        ks = _timed(lambda: pl.solve(sc, p, want_xi=False), 5, flush, stream)
        flops = algorithmic_flops_per_sample_iter(prm.m, prm.n_coef, sc.n_obs) * B * prm.inner_iters
        rows.append({"B": B, "ms_per_cycle": statistics.median(ms),
                     "sample_iters_per_s": B * prm.inner_iters * prm.outer_iters / (statistics.median(ms) / 1e3),
                     "solve_ms": statistics.median(ks),
                     "solve_tflops": flops / (statistics.median(ks) * 1e-3) / 1e12})
        pl.close()
    # the plain float64 path on the smallest point, one cycle (it is ~100x slower)
    prm, sc, _ = sg.workload(4, B=1024)
    pf = Planner(prm, prec="fp64", max_obs=32, max_samples=1024)
    pf.upload([sc])
    pf.set_state(0, seed=7, step=0)
    pf.step_resident([1024])
    ms64 = _timed(lambda: pf.step_resident([1024]), 1, flush, stream,
                  prep=lambda i: pf.set_state(0, seed=7, step=1 + i))[0]
    pf.close()
    plain = {"B": 1024, "ms_per_cycle": ms64,
             "sample_iters_per_s": 1024 * prm.inner_iters * prm.outer_iters / (ms64 / 1e3),
             "fp32_speedup": ms64 / rows[0]["ms_per_cycle"]}
    print(json.dumps({"metric": METRIC, "workload": "scale", "unit": UNIT, "dtype": "f32",
                      "config": {"workload": "6 lanes, N=30, m=200, n=16, K=100, L=5"},
                      "rows": rows, "plain_fp64": plain}))


def serving_arm(args):
    print(json.dumps(serve(args.rate, args.serve_seconds, args.serve_episodes, args.serve_b,
                           args.executors)))


def serve(rate, seconds, n_ep=64, serve_b=(512, 2048), executors=16):
    """Served MPC loop: Poisson arrivals of cycle requests at `rate` per second
    over rolling 50-cycle episodes (N 4..24, B 512..2048, horizon in
    {80, 100, 125, 150}); each episode advances its scene by plan_advance after
    every result.  Each episode (vehicle) has at most one cycle in flight: an
    arrival that finds every episode busy waits in a FIFO until one is idle, so
    no arrival is dropped.  Latencies: `server` = submission to completion inside
    the server (its own queue included); `e2e` = arrival to completion (the wait
    for an idle episode included).  Arrivals stop after --serve-seconds; the run
    ends when every arrival has completed."""
    import collections
    import numpy as np
    from paper_2212_02224_gb300 import scenegen as sg
    from paper_2212_02224_gb300.planner import Server, advance
    prm, _, _ = sg.workload(1)
    srv = Server(prm, max_obs=24, max_samples=16384, max_scenes=32, max_executors=executors,
                 device_budget=16 << 30, max_episodes=4096)
    rng = np.random.default_rng(11)
    s = sg.Stream(4242)
    eps = []
    for e in range(n_ep):
        sc = sg.make_scene(50000 + e, n_lanes=4, n_obs=int(s.integers(4, 24, 1)[0]))
        eps.append(dict(id=e, scene=sc, B=int(s.integers(serve_b[0], serve_b[1], 1)[0]),
                        m=int(rng.choice([80, 100, 125, 150])), cycle=0, busy=False, ticket=None,
                        t_arr=0.0))
    # warm the executors (one per horizon) before timing
    for m in (80, 100, 125, 150):
        srv.wait(srv.submit(eps[0]["scene"], 512, m=m, episode=10**9 + m, seed=1))
        srv.end_episode(10**9 + m)
    lat, lat_e2e, done_units = [], [], 0
    by_ticket = {}
    waiting = collections.deque()          # arrival times waiting for an idle episode
    max_waiting = 0
    t0 = time.perf_counter()
    next_arrival = t0
    duration = seconds
    offered = submitted = completed = 0
    next_ep_id = n_ep
    while True:
        now = time.perf_counter()
        if now - t0 > duration and not by_ticket and not waiting:
            break
        while now >= next_arrival and next_arrival - t0 <= duration:
            waiting.append(next_arrival)     # every arrival that is due
            offered += 1
            next_arrival += rng.exponential(1.0 / rate)
        max_waiting = max(max_waiting, len(waiting))
        if waiting:
            idle = [e for e in eps if not e["busy"]]
            while waiting and idle:
                e = idle.pop(int(rng.integers(len(idle))))
                e["t_arr"] = waiting.popleft()
                e["ticket"] = srv.submit(e["scene"], e["B"], m=e["m"], episode=e["id"], seed=e["id"])
                e["busy"] = True
                by_ticket[e["ticket"]] = e
                submitted += 1
        # block on the server's completions until the next arrival is due
        wait_s = next_arrival - time.perf_counter() if next_arrival - t0 <= duration else 0.005
        got = srv.poll_any(int(max(0.0, min(wait_s, 0.005)) * 1e6))
        while got is not None:
            ticket, r = got
            t_done = time.perf_counter()
            e = by_ticket.pop(ticket)
            e["busy"] = False
            completed += 1
            lat.append(r["latency_us"] / 1e3)
            lat_e2e.append((t_done - e["t_arr"]) * 1e3)
            done_units += e["B"] * prm.inner_iters * prm.outer_iters
            e["cycle"] += 1
            if e["cycle"] >= 50:              # episode over: a new vehicle takes the slot
                srv.end_episode(e["id"])
                e["id"], e["cycle"] = next_ep_id, 0
                next_ep_id += 1
                e["scene"] = sg.make_scene(60000 + e["id"], n_lanes=4,
                                           n_obs=int(s.integers(4, 24, 1)[0]))
            else:
                e["scene"] = advance(prm, e["scene"], r["xi"])
            got = srv.poll_any(0)
    wall = time.perf_counter() - t0
    info = srv.info()
    srv.close()

    def pct(v, q):
        return float(np.percentile(v, q))

    return {
        "metric": METRIC, "workload": "serving", "rate_req_s": rate,
        "achieved_req_s": completed / wall, "value": done_units / wall, "unit": UNIT,
        "latency_ms": {"p50": pct(lat_e2e, 50), "p99": pct(lat_e2e, 99), "mean": float(np.mean(lat_e2e)),
                       "basis": "arrival to completion: the wait for an idle episode and the "
                                "server's queue included"},
        "server_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99),
                              "basis": "submission to completion inside the server"},
        "offered": offered, "submitted": submitted, "completed": completed, "dropped": 0,
        "max_waiting_for_episode": max_waiting, "wall_s": wall,
        "waves": info["waves"], "max_wave": info["max_wave"], "executors": info["executors"],
        "dtype": "f32",
        "config": {"workload": "Poisson arrivals over %d rolling 50-cycle episodes, N 4..24, "
                               "B %d..%d, m in {80,100,125,150}, K=100, L=5, elites 150/50"
                               % (n_ep, serve_b[0], serve_b[1])}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="leave out the scale point and the batched step of the default line")
    ap.add_argument("--latency-cycles", type=int, default=1000,
                    help="cycles of the latency run after 50 warm-up cycles (0: none)")
    ap.add_argument("--workload", default="dense", choices=["dense", "batched", "scale", "serving"])
    ap.add_argument("--rate", type=float, default=200.0, help="serving: requests per second")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--executors", type=int, default=16, help="serving: planner contexts")
    ap.add_argument("--serve-b", type=int, nargs=2, default=[512, 2048],
                    help="serving: range of samples per request")
    ap.add_argument("--serve-episodes", type=int, default=64,
                    help="serving: concurrent episodes (vehicles), one cycle in flight each")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "scale":
        scale_arm(args)
    elif args.workload == "serving":
        serving_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()

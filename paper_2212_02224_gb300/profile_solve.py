"""Repeated lower-level solves or MPC cycles of one workload, for profilers and
for timing comparisons.

    python -m paper_2212_02224_gb300.profile_solve --prec fp32 --shape 2 1 --reps 3
    python -m paper_2212_02224_gb300.profile_solve --prec tf32x3 --reps 1
    python -m paper_2212_02224_gb300.profile_solve --workload scale --samples 8192 \\
        --persistent on --reps 2
    python -m paper_2212_02224_gb300.profile_solve --workload batched --shape 1 4 --time 5
    python -m paper_2212_02224_gb300.profile_solve --shape 1 7 --cycles 300

Without --time or --cycles, each call solves the same samples `reps` times on the
current device and synchronises, so a profiler can skip the warm-up launches
and capture one solve of one kernel.  --time N times N solves and --cycles N
times N graph-captured MPC cycles (Alg. 1, each a fresh planning call), with
CUDA events on the launching stream after `reps` warm-up runs and a 256 MiB
write between timed runs (larger than L2); they print one JSON line with the
median and the minimum in milliseconds.

Workloads: dense (B = 1000 by default; 4 lanes, 12 obstacles, m = 100, n = 11,
K = 100), scale (6 lanes, 30 obstacles, m = 200, n = 16, K = 100) and batched
(256 scenes, N ~ U{4..20}, B ~ U{256..2048}, m = 100, n = 11, K = 100; --samples
is ignored).  --persistent sets the launch form of the fused FP32 kernel.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np
import torch

from . import scenegen as sg
from .planner import Planner


def _timed(run, n, prep=None):
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ts = []
    for i in range(n):
        if prep:
            prep(i)
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return {"median_ms": statistics.median(ts), "min_ms": min(ts), "n": n}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--shape", type=int, nargs=2, default=None,
                    help="fused FP32 kernel shape: warps per sample, samples per CTA")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--samples", type=int, default=1000)
    ap.add_argument("--workload", default="dense", choices=["dense", "scale", "batched"])
    ap.add_argument("--persistent", default="auto", choices=["auto", "off", "on"])
    ap.add_argument("--time", type=int, default=0, help="time this many solves")
    ap.add_argument("--cycles", type=int, default=0, help="time this many MPC cycles")
    args = ap.parse_args(argv)
    if args.workload == "batched":
        prm, scenes, Bs = sg.batched_workload(S=256)
        max_obs = 20
    else:
        prm, sc, _ = sg.workload(1 if args.workload == "dense" else 4)
        scenes, Bs = [sc], [args.samples]
        max_obs = 16 if args.workload == "dense" else 32
    total = sum(Bs)
    p = torch.tensor(np.concatenate([sg.make_samples(303 + i, scenes[i], Bs[i], prm.n_seg)
                                     for i in range(len(scenes))]),
                     dtype=torch.float64, device="cuda")
    pl = Planner(prm, prec=args.prec, max_obs=max_obs, max_samples=total, max_scenes=len(scenes))
    if args.shape:
        pl.set_tuning(*args.shape)
    if args.prec == "fp32":
        pl.set_persistent(args.persistent)

    def solve():
        if len(scenes) == 1:
            pl.solve(scenes[0], p, want_xi=False)
        else:
            pl.solve_batch(scenes, Bs, p)

    if args.cycles:
        pl.upload(scenes)

        def fresh(i):
            for k in range(len(scenes)):
                pl.set_state(k, seed=1234 + k, step=i)

        for i in range(args.reps):
            fresh(i)
            pl.step_resident(Bs)
        out = _timed(lambda: pl.step_resident(Bs), args.cycles, prep=fresh)
        print(json.dumps({"what": "cycle", "workload": args.workload, "samples": total, **out}))
    elif args.time:
        for _ in range(args.reps):
            solve()
        out = _timed(solve, args.time)
        print(json.dumps({"what": "solve", "workload": args.workload, "samples": total, **out}))
    else:
        for _ in range(args.reps):
            solve()
        torch.cuda.synchronize()
        print(f"{args.reps} solves of {total} samples ({args.prec}) done")
    pl.close()


if __name__ == "__main__":
    main()

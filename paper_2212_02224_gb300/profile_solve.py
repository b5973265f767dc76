"""Repeated lower-level solves of one workload, for profilers.

    python -m paper_2212_02224_gb300.profile_solve --prec fp32 --shape 2 1 --reps 3
    python -m paper_2212_02224_gb300.profile_solve --prec tf32x3 --reps 1
    python -m paper_2212_02224_gb300.profile_solve --workload scale --samples 8192 \
        --persistent on --reps 2

Each call solves the same samples `reps` times on the current device and
synchronises, so a profiler can skip the warm-up launches and capture one solve
of one kernel.  Workloads: dense (B = 1000 by default; 4 lanes, 12 obstacles,
m = 100, n = 11, K = 100) and scale (6 lanes, 30 obstacles, m = 200, n = 16,
K = 100).  --persistent sets the launch form of the fused FP32 kernel.
"""
from __future__ import annotations

import argparse

import torch

from . import scenegen as sg
from .planner import Planner


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--shape", type=int, nargs=2, default=None,
                    help="fused FP32 kernel shape: warps per sample, samples per CTA")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--samples", type=int, default=1000)
    ap.add_argument("--workload", default="dense", choices=["dense", "scale"])
    ap.add_argument("--persistent", default="auto", choices=["auto", "off", "on"])
    args = ap.parse_args(argv)
    prm, sc, _ = sg.workload(1 if args.workload == "dense" else 4)
    B = args.samples
    p = torch.tensor(sg.make_samples(303, sc, B, prm.n_seg), dtype=torch.float64, device="cuda")
    pl = Planner(prm, prec=args.prec, max_obs=16 if args.workload == "dense" else 32, max_samples=B)
    if args.shape:
        pl.set_tuning(*args.shape)
    if args.prec == "fp32":
        pl.set_persistent(args.persistent)
    for _ in range(args.reps):
        pl.solve(sc, p, want_xi=False)
    torch.cuda.synchronize()
    pl.close()
    print(f"{args.reps} solves of {B} samples ({args.prec}) done")


if __name__ == "__main__":
    main()

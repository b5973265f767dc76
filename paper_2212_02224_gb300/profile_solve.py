"""Repeated lower-level solves of the dense-traffic workload, for profilers.

    python -m paper_2212_02224_gb300.profile_solve --prec fp32 --shape 2 1 --reps 3
    python -m paper_2212_02224_gb300.profile_solve --prec tf32x3 --reps 1

Each call solves the same B = 1000 samples (4 lanes, 12 obstacles, m = 100,
n = 11, K = 100) `reps` times on the current device and synchronises, so a
profiler can skip the warm-up launches and capture one solve of one kernel.
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
    args = ap.parse_args(argv)
    prm, sc, _ = sg.workload(1)
    B = args.samples
    p = torch.tensor(sg.make_samples(303, sc, B, prm.n_seg), dtype=torch.float64, device="cuda")
    pl = Planner(prm, prec=args.prec, max_obs=16, max_samples=B)
    if args.shape:
        pl.set_tuning(*args.shape)
    for _ in range(args.reps):
        pl.solve(sc, p, want_xi=False)
    torch.cuda.synchronize()
    pl.close()
    print(f"{args.reps} solves of {B} samples ({args.prec}) done")


if __name__ == "__main__":
    main()

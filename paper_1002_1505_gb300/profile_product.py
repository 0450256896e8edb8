"""Per-pass timing of the FFT-convolution product A.P for one of the bench workloads.

    python -m paper_1002_1505_gb300.profile_product --workload prism48 [--schedule plane512] [--iters 20]
                                                   [--c128 | --df] [--orientations K]

Sets up the workload's target, beams, Green tensor and polarizability, then
times `iters` products of every RHS with CUDA events between the passes
(dda_profile_matvec) and prints the schedule and the mean time of each pass:
complex64 by default, complex128 with --c128, the double-float product of the
true residuals with --df; --orientations K keeps the first K orientations of the workload (a smaller
batch on the same grid, for profiler captures that must stay small).
Small and short on purpose: it is the command to run under ncu for one kernel
(`-k regex:k_yz_plane -s 2 -c 1`).
"""
from __future__ import annotations

import argparse
import os


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ellipsoid64",
                    choices=["sphere12", "ellipsoid64", "prism48", "hexprism160", "au_block"])
    ap.add_argument("--schedule", default=None,
                    help="pin the product schedule (generic, fast5, plane512, plane768, cluster2, cluster4)")
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--c128", action="store_true")
    ap.add_argument("--df", action="store_true", help="complex128 product in double-float arithmetic")
    ap.add_argument("--orientations", type=int, default=0, help="first K orientations only (0 = all)")
    args = ap.parse_args()
    if args.schedule:
        os.environ["DDA_SCHEDULE"] = args.schedule
    from . import dda as D
    from . import workloads as W
    w = {"sphere12": W.SPHERE12, "ellipsoid64": W.ELLIPSOID64, "prism48": W.PRISM48,
         "hexprism160": W.HEXPRISM160, "au_block": W.AU_BLOCK}[args.workload]
    if args.orientations > 0:
        import dataclasses
        w = dataclasses.replace(w, orientations=w.orientations[:args.orientations])
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    dt = D.DDA_C128DF if args.df else (D.DDA_C128 if args.c128 else D.DDA_C64)
    ms = D.dda_profile_matvec(ctx, ctx.nrhs, dt, args.iters)
    info = D.dda_schedule_info(ctx, dt)
    print(f"{w.name}: N={ctx.n} box={ctx.box} rhs={ctx.nrhs} schedule(passes, fast, threads, tuned_nrhs, "
          f"ctas_per_plane)={info} pass ms={[round(float(v), 4) for v in ms]} total={float(ms.sum()):.4f} ms")
    ctx.close()


if __name__ == "__main__":
    main()

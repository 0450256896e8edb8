#!/usr/bin/env python
"""Benchmark of the DDA hot path on GB300: FFT-convolution A.P throughput and
solve time per orientation at residual 1e-5, against the plain FP64 GPU solve.

One step = the whole path for one batch: incident beams and polarizabilities
for every RHS, the FP64 Fourier-space Green tensor, the batched BiCGstab solve
(complex64 iterations refined against FP64-accurate true residuals, whose product runs in
double-float arithmetic) to |E - A P|/|E| <= 1e-5,
and the efficiencies plus Mueller elements.  The target's site list is resident
on the device before the timed region (it is the step's input).

value = A.P products per second (one product = A applied to one RHS vector, any
precision, counted per RHS: the products a batch skips for RHS whose solve has
finished are not counted) summed over all ranks; --gpus N runs N independent
replicas.
--impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1002_1505_gb300 import workloads as W  # noqa: E402

WORKLOADS = {"ellipsoid64": W.ELLIPSOID64, "prism48": W.PRISM48, "hexprism160": W.HEXPRISM160,
             "sphere12": W.SPHERE12, "au_block": W.AU_BLOCK, "mixed": None}
MUELLER_DIRS = [(0.0, 0.0), (math.pi / 2, 0.0), (math.pi, 0.0), (math.pi / 2, math.pi / 2)]
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
METRIC = "FFT-conv A.P matvecs/s and solve time/orientation @1e-5 residual vs plain GPU"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(w, n, box, pad, ws):
    """The config object of the JSON line, the same for both arms: workload w with n sites in its
    box on the padded grid, orientations sharded over ws ranks (rank 0's share is the one named)."""
    from paper_1002_1505_gb300 import replicas
    a_o, b_o = replicas.shard(len(w.orientations), 0, ws)
    n_ori = b_o - a_o
    nrhs = n_ori * w.iorth
    return {"workload": w.name, "n_dipoles": int(n), "box": [int(v) for v in box], "pad": [int(v) for v in pad],
            "nrhs": nrhs * ws, "n_orientations": len(w.orientations), "tol": 1e-5,
            "solver": "BiCGstab, complex64 + FP64-accurate refinement",
            "true_residual": "double-float product (FP32 pairs, within 1e-12 of FP64) where the grid "
                             "has compile-time kernels, else complex128",
            "l2": "flushed (512 MB write) before every step",
            "parallelism": f"replicas x{ws}: orientations sharded over ranks, "
                           f"{n_ori} orientations ({nrhs} RHS) per rank"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(sched_passes: int, n: int, box, pad, nrhs: int, csize: int, fast: bool = True):
    """Bytes per launch of each pass (byte model of the 3-pass / 5-pass schedule) and kernel names."""
    nx, ny, nz = box
    px, py, pz = pad
    xrow = px * ny * nz            # spectrum after the x pass (per component)
    yrow = px * py * nz            # after the y pass (5-pass only)
    ghat = 6 * px * py * pz        # Fourier-space tensor, read once per batch
    b3 = 3 * nrhs
    if sched_passes == 3:
        per = [b3 * (n + xrow), b3 * 2 * xrow + ghat, b3 * (xrow + n)]
        names = ["k_x_fwd", "k_yz_plane", "k_x_inv"] if fast else ["k_xfwd", "k_yzplane", "k_xinv"]
    else:
        per = [b3 * (n + xrow), b3 * (xrow + yrow), b3 * 2 * yrow + ghat, b3 * (yrow + xrow), b3 * (xrow + n)]
        names = (["k_x_fwd", "k_y_rows(fwd)", "k_z_cols", "k_y_rows(inv)", "k_x_inv"] if fast else
                 ["k_xfwd", "k_fft_rows(y fwd)", "k_zconv", "k_fft_rows(y inv)", "k_xinv"])
    return [v * csize for v in per], names


# FP32 issue roofline of the GB300 SMs: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def algorithmic_flops(sched_passes: int, box, pad, nrhs: int):
    """FP32 flops per launch of each pass: 5 L log2 L per complex FFT of length L (no credit for the
    pruned zero halves), 66 flops per voxel for the 3x3 symmetric Fourier-space multiply."""
    nx, ny, nz = box
    px, py, pz = pad
    fft = lambda L: 5.0 * L * math.log2(L)
    xl = 3 * ny * nz * fft(px)                  # x lines, one direction
    yl = 3 * nz * px * fft(py)
    zl = 3 * px * py * fft(pz)
    gm = 66.0 * px * py * pz
    if sched_passes == 3:
        per = [xl, 2 * yl + 2 * zl + gm, xl]
    else:
        per = [xl, yl, 2 * zl + gm, yl, xl]
    return [v * nrhs for v in per]


def cufft_product_ms(box, pad, nrhs: int, stream, iters: int = 10):
    """Timed comparison only: the same zero-padded convolution with cuFFT (torch.fft) and torch
    element-wise ops for the 3x3 Fourier-space multiply, on box-shaped input (no site gather or
    scatter, no alpha^{-1} term), CUDA events on the launching stream."""
    import torch
    nx, ny, nz = box
    px, py, pz = pad
    g = torch.randn((6, pz, py, px), dtype=torch.complex64, device="cuda")
    v = torch.randn((nrhs, 3, nz, ny, nx), dtype=torch.complex64, device="cuda")
    idx = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]

    def prod():
        f = torch.fft.fftn(v, s=(pz, py, px), dim=(-3, -2, -1))
        u = torch.stack([g[idx[a][0]] * f[:, 0] + g[idx[a][1]] * f[:, 1] + g[idx[a][2]] * f[:, 2]
                         for a in range(3)], dim=1)
        return torch.fft.ifftn(u, dim=(-3, -2, -1))[..., :nz, :ny, :nx]

    def ffts_only():
        f = torch.fft.fftn(v, s=(pz, py, px), dim=(-3, -2, -1))
        return torch.fft.ifftn(f, dim=(-3, -2, -1))

    out = []
    for fn in (prod, ffts_only):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(iters):
            fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1) / iters)
    del g, v
    torch.cuda.empty_cache()
    return out


def run_reference(args, w):
    """Oracle arm: the FP64 CPU FFT-convolution product of the same workload."""
    from oracle import dda as odda
    t0 = time.time()
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations, e01_lf=w.e01,
                              iorth=w.iorth, pad=w.pad)
    from oracle import interaction as oint
    ghat = oint.green_fft(prob.target.box, prob.pad, prob.kd, workers=-1)
    rng = np.random.default_rng(1)
    p = rng.standard_normal((3, prob.target.n)) + 1j * rng.standard_normal((3, prob.target.n))
    # a bounded sample of the workload's products per step: two RHS on the small grids, one on the
    # multi-million-point grids (each FP64 product there takes seconds on the host cores)
    per_step = min(len(prob.rhs), 2 if np.prod(prob.pad) < 4_000_000 else 1)

    def step():
        for b in range(per_step):
            odda.apply_a(prob, b, p, "fft", ghat=ghat, workers=-1)

    for _ in range(args.warmup):
        step()
    t = time.time()
    for _ in range(args.steps):
        step()
    dt = time.time() - t
    value = args.steps * per_step / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": workload_config(w, prob.target.n, prob.target.box, prob.pad, dist_env()[0]),
            "cpu_baseline": {"value": value, "unit": "matvecs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} FFT-convolution products A.P (FP64, scipy.fft, workers={cores}) "
                                       f"per step on {w.name}"},
            "e2e": {"value": value, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": t - t0}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, budget_s=15.0):
    """The oracle's FFT-convolution product timed on the host cores, bounded sample."""
    from oracle import dda as odda
    from oracle import interaction as oint
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations[:1], e01_lf=w.e01,
                              iorth=1, pad=w.pad)
    ghat = oint.green_fft(prob.target.box, prob.pad, prob.kd, workers=-1)
    rng = np.random.default_rng(2)
    p = rng.standard_normal((3, prob.target.n)) + 1j * rng.standard_normal((3, prob.target.n))
    odda.apply_a(prob, 0, p, "fft", ghat=ghat, workers=-1)
    count, t = 0, time.time()
    while time.time() - t < budget_s:
        odda.apply_a(prob, 0, p, "fft", ghat=ghat, workers=-1)
        count += 1
    dt = time.time() - t
    cores = os.cpu_count()
    return {"value": count / dt, "unit": "matvecs/s", "cores": cores, "kind": "oracle",
            "sample": f"{count} FP64 FFT-convolution products A.P (one RHS each, scipy.fft workers={cores}) on "
                      f"{w.name}, {dt:.1f} s"}


def run_mixed(args):
    """Uneven mixed batch (spheres D = 16..64, three cylinders; |m| kd = 0.5; 2 orientations x 2
    polarizations each) solved concurrently with dda_solve_batch, against the same targets solved
    one after another."""
    import torch
    from paper_1002_1505_gb300 import dda as D
    ws = W.mixed_batch()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctxs, kds = [], []
    for w in ws:
        c = D.Context(0, stream)
        c.dda_setup_shape(w.shape, w.shpar)
        ctxs.append(c)
        kds.append(0.5 / abs(w.m))
    ps = [torch.zeros((len(w.orientations) * w.iorth, 3, c.n), dtype=torch.complex128, device="cuda")
          for w, c in zip(ws, ctxs)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def setup_all():
        for w, c, kd in zip(ws, ctxs, kds):
            c.dda_set_incident(kd, w.orientations, [[q[0], q[1]] for q in w.e01], w.iorth)
            c.dda_build_green_fft()
            c.dda_set_polarizability(w.prescription, w.m)

    def step(concurrent=True):
        setup_all()
        if concurrent:
            reps, sts, overall = D.dda_solve_batch(ctxs, ps, precision="MIXED", tol=1e-5, maxit=3000)
            assert overall == D.DDA_OK, sts
        else:
            reps = [c.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000)[0] for c, p in zip(ctxs, ps)]
        for c, p in zip(ctxs, ps):
            c.dda_cross_sections(p)
        return sum(x["matvecs"] for r in reps for x in r), reps

    def timed(k, concurrent):
        tot, mv = 0.0, 0
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m, reps = step(concurrent)
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
            mv += m
        return tot * 1e3, mv, reps

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(0)
    k0 = D.dda_kernel_launches()
    ms, mv, reps = timed(args.steps, True)
    launches = D.dda_kernel_launches() - k0
    clk = clocks.stop()
    seq_ms, _, _ = timed(max(1, args.steps // 2), False)
    seq_ms /= max(1, args.steps // 2)
    n_ori = sum(len(w.orientations) for w in ws)
    line = {"metric": METRIC, "value": mv / (ms / 1e3), "unit": "matvecs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": "mixed batch: " + ", ".join(w.name for w in ws),
                       "n_dipoles": [c.n for c in ctxs], "nrhs_total": sum(len(r) for r in reps),
                       "tol": 1e-5, "l2": "flushed (512 MB write) before every step", "parallelism": "replicas x1"},
            "solve_ms_per_orientation": ms / args.steps / n_ori,
            "sequential_ms_per_step": seq_ms, "concurrency_speedup": seq_ms / (ms / args.steps),
            "schedules": [D.dda_schedule_info(c, D.DDA_C64) for c in ctxs],
            "gpu_launches": int(launches), "clocks": clk,
            "note": "wall-clock per step (host threads drive one stream per target)"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="hexprism160", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-reps", type=int, default=1)
    ap.add_argument("--plain-orientations", type=int, default=0,
                    help="orientations the plain FP64 comparator solves (0 = all; default 2 on the hexagonal "
                         "prism, whose plain solve takes seconds per orientation)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="timed steps of the end-to-end leg (0 = min(steps, as many as fit in ~30 s))")
    ap.add_argument("--unet-problems", type=int, default=2048,
                    help="random training problems for the in-bench network of the warm-start leg (0 = no network)")
    ap.add_argument("--unet-steps", type=int, default=4000)
    ap.add_argument("--warm-start", default="auto", choices=["auto", "on", "off"],
                    help="also time the solve warm-started from the network-free guess alpha E_inc "
                         "(auto = on for the hexagonal prism)")
    ap.add_argument("--orientations", type=int, default=0,
                    help="use only the first N orientations of the workload (smaller profiling runs)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if w is None:
        run_mixed(args)
        return
    if args.orientations > 0:
        import dataclasses
        w = dataclasses.replace(w, name=f"{w.name}[:{args.orientations}]",
                                orientations=w.orientations[:args.orientations])
    ws, rank, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import torch
    import torch.distributed as dist
    from paper_1002_1505_gb300 import dda as D
    from paper_1002_1505_gb300 import replicas

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = D.Context(local, stream)
    n, box = ctx.dda_setup_shape(w.shape, w.shpar)
    kd, _ = ctx.dda_kd_from_x(w.x)
    e01 = [[c[0], c[1]] for c in w.e01]
    # replica mode: each rank solves its contiguous share of the orientations (independent systems
    # sharing the target; nothing is exchanged on the data path)
    a_o, b_o = replicas.shard(len(w.orientations), rank, ws)
    my_ori = list(w.orientations[a_o:b_o])
    n_ori = len(my_ori)
    if n_ori == 0:
        raise SystemExit(f"rank {rank}: no orientations left for this rank ({len(w.orientations)} over {ws})")
    nrhs = n_ori * w.iorth
    p = torch.zeros((nrhs, 3, n), dtype=torch.complex128, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(precision="MIXED", use_graph=True, ori=None, warm=None):
        ori = my_ori if ori is None else ori
        pp = p[:len(ori) * w.iorth]
        ctx.dda_set_incident(kd, ori, e01, w.iorth)
        ctx.dda_build_green_fft(w.pad)
        ctx.dda_set_polarizability(w.prescription, w.m)
        if warm is not None:
            pp.copy_(warm(ctx))
        reps, _ = ctx.dda_solve(pp, solver="BICGSTAB", precision=precision, tol=1e-5, maxit=3000,
                                use_graph=use_graph, warm_start=warm is not None)
        q, mm = ctx.dda_cross_sections(pp, MUELLER_DIRS if w.iorth == 2 else None)
        return reps, q

    def timed(nsteps, **kw):
        total, mv, last = 0.0, 0, None
        for _ in range(nsteps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps, q = step(**kw)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            mv += sum(r["matvecs"] for r in reps)  # products actually applied to each RHS
            last = (reps, q)
        return total, mv, last

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    k0 = D.dda_kernel_launches()
    total_ms, matvecs, (reps, q) = timed(args.steps)
    launches = D.dda_kernel_launches() - k0
    torch.cuda.synchronize()
    clk = clocks.stop()
    my_ms = total_ms
    if ws > 1:
        total_ms, matvecs = replicas.reduce_max_sum(total_ms, float(matvecs))
    value = matvecs / (total_ms / 1e3)
    ms_step = total_ms / args.steps
    # the guide's orientation average (equal weights for the seeded uniform orientations), gathered
    # from every rank's share
    w_all = np.full(len(w.orientations), 1.0 / len(w.orientations))
    q_avg = replicas.orientation_average_sharded(q[:, :3], w_all[a_o:b_o], w.iorth,
                                                 group=None) if ws > 1 else D.dda_orientation_average(
                                                     q[:, :3], w_all[a_o:b_o], w.iorth)

    # plain FP64 GPU comparator: complex128 BiCGstab, no refinement, one launch per kernel, on the
    # first few orientations (it takes seconds per orientation on the large grids)
    n_plain = args.plain_orientations or (2 if np.prod(w.pad or (1,)) > 8_000_000 else n_ori)
    plain_ori = my_ori[:max(1, min(n_plain, n_ori))]
    plain_ms, plain_mv, (preps, pq) = timed(args.plain_reps, precision="C128", use_graph=False, ori=plain_ori)
    plain_ms_per_ori = plain_ms / args.plain_reps / len(plain_ori)
    # back to every orientation of this rank (the context's RHS count follows the last set-up)
    ctx.dda_set_incident(kd, my_ori, e01, w.iorth)
    ctx.dda_build_green_fft(w.pad)
    ctx.dda_set_polarizability(w.prescription, w.m)

    # warm-started solves (config 5: the same mixed-precision solve from an initial guess): the
    # network-free local-field guess P0 = alpha E_inc, and the learned network's guess when a short
    # in-bench training is asked for; iterations and time at the same final residual as the cold solve
    warm_report = None
    want_warm = args.warm_start == "on" or (args.warm_start == "auto" and w is WORKLOADS["hexprism160"])
    if want_warm and ws == 1:
        from paper_1002_1505_gb300 import warmstart as WS
        warm_report = {"cold": {"iterations": int(sum(r["iters"] for r in reps)), "ms_per_orientation": ms_step / n_ori,
                                "max_true_rel_resid": float(max(r["true_rel_resid"] for r in reps))}}
        grid = WS.grid_dims(box)
        guesses = {"alpha_einc": lambda c: WS.local_field_guess(c, grid)}
        if args.unet_problems > 0:
            t0 = time.perf_counter()
            net = WS.train_quick(args.unet_problems, args.unet_steps)
            warm_report["network_training_s"] = time.perf_counter() - t0
            warm_report["network_training"] = {"problems": args.unet_problems, "steps": args.unet_steps,
                                               "max_box": 16, "params": int(net.nparams)}
            guesses["network"] = lambda c: WS.warm_guess(c, net, grid, chunk=2)
        for nm, fn in guesses.items():
            wms, wmv, (wreps, _) = timed(1, warm=fn)
            warm_report[nm] = {"iterations": int(sum(r["iters"] for r in wreps)), "ms_per_orientation": wms / n_ori,
                               "max_true_rel_resid": float(max(r["true_rel_resid"] for r in wreps)),
                               "includes": "guess construction + solve + observables"}

    # end to end through the C ABI with host buffers: site list in, solution P and Q out
    sites, origin = ctx.dda_get_sites()
    h_sites = np.ascontiguousarray(sites)
    h_p = torch.empty((nrhs, 3, n), dtype=torch.complex128, pin_memory=True)
    ctx2 = D.Context(local, stream)
    e2e_steps = args.e2e_steps or max(2, min(args.steps, int(30e3 / max(ms_step, 1.0))))
    e2e_ms = 0.0
    e2e_mv = 0
    for i in range(1 + e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.dda_setup_target(h_sites, origin=origin)
        ctx2.dda_set_incident(kd, my_ori, e01, w.iorth)
        ctx2.dda_build_green_fft(w.pad)
        ctx2.dda_set_polarizability(w.prescription, w.m)
        p2 = torch.zeros((nrhs, 3, n), dtype=torch.complex128, device="cuda")
        r2, _ = ctx2.dda_solve(p2, precision="MIXED", tol=1e-5, maxit=3000)
        q2, _ = ctx2.dda_cross_sections(p2, MUELLER_DIRS if w.iorth == 2 else None)
        h_p.copy_(p2, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        dt = time.perf_counter() - t0
        if i >= 1:
            e2e_ms += dt * 1e3
            e2e_mv += sum(r["matvecs"] for r in r2)
    ctx2.close()
    del p2
    if ws > 1:
        e2e_ms, e2e_mv = replicas.reduce_max_sum(e2e_ms, float(e2e_mv))
    e2e_value = e2e_mv / (e2e_ms / 1e3)
    h2d = h_sites.nbytes + 3 * n_ori * 8 + 48
    d2h = h_p.numel() * 16 + q2.nbytes

    # dominant pass of the product: CUDA events between passes on the launching stream
    ms_pass = D.dda_profile_matvec(ctx, nrhs, D.DDA_C64, iters=20)
    sched = D.dda_schedule_info(ctx, D.DDA_C64)
    cs = 8
    pad = w.pad if w.pad else tuple(int(v) for v in np.array(box) * 2)
    abytes, names = algorithmic_bytes(len(ms_pass), n, box, pad, nrhs, cs, fast=bool(sched[1]))
    dom = int(np.argmax(ms_pass))
    peak, peak_kind = peaks()
    achieved = abytes[dom] / (ms_pass[dom] * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as fh:
            tj = json.load(fh)
        key = f"{names[dom]}@{w.name}"
        traffic = tj.get(key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": names[dom], "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": abytes[dom], "ms_per_launch": ms_pass[dom],
                "passes_ms": {nm: float(v) for nm, v in zip(names, ms_pass)},
                "schedule": {"passes": sched[0], "compile_time_kernels": bool(sched[1]),
                             "plane_threads": sched[2], "tuned_for_nrhs": sched[3], "ctas_per_plane": sched[4],
                             "x_tile_rows": sched[5], "bulk_staged_plane": bool(sched[6]),
                             "x_components_per_cta": sched[7], "z_register_fused": bool(sched[8])},
                "product_ms": float(np.sum(ms_pass))}
    # the FP64-accurate product of the true residuals: complex128 on the FP64 units against
    # double-float arithmetic on the FP32 units (the one the mixed solve uses where it exists)
    fp64_products = {}
    for nm, dt in (("complex128", D.DDA_C128), ("double_float", D.DDA_C128DF)):
        try:
            fp64_products[nm] = float(np.sum(D.dda_profile_matvec(ctx, nrhs, dt, iters=5)))
        except D.DDAError as exc:
            fp64_products[nm] = str(exc).splitlines()[0]
    flops = algorithmic_flops(len(ms_pass), box, pad, nrhs)
    tfl = flops[dom] / (ms_pass[dom] * 1e-3) / 1e12
    roofline["alu"] = {"bound": "fp32 issue", "achieved": tfl, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": tfl / FP32_PEAK_TFLOPS, "flops_per_launch": flops[dom],
                       "peak_kind": "nominal: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    try:
        cu_ms, cu_fft_ms = cufft_product_ms(box, pad, nrhs, stream)
        roofline["cufft_compare"] = {"cufft_product_ms": cu_ms, "cufft_ffts_only_ms": cu_fft_ms,
                                     "ours_product_ms": float(np.sum(ms_pass)),
                                     "ratio": cu_ms / float(np.sum(ms_pass)),
                                     "note": "torch.fft (cuFFT) zero-padded 3-D FFT + inverse of 3 components "
                                             "(+ torch 3x3 multiply for cufft_product_ms) on box-shaped input"}
    except RuntimeError as exc:  # e.g. out of memory on the largest grids
        roofline["cufft_compare"] = {"error": str(exc).splitlines()[0]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": workload_config(w, n, box, pad, ws),
            "solve_ms_per_orientation": ms_step / n_ori,
            "plain_fp64_solve_ms_per_orientation": plain_ms_per_ori,
            "plain_fp64_orientations_timed": len(plain_ori),
            "speedup_vs_plain_fp64": plain_ms_per_ori / (ms_step / n_ori),
            "iterations": [r["iters"] for r in reps], "plain_iterations": [r["iters"] for r in preps],
            "true_rel_resid": [r["true_rel_resid"] for r in reps],
            "true_residual_product_ms": fp64_products,
            "Q": {"Qext": q[:, 0].tolist(), "Qabs": q[:, 1].tolist(), "Qsca": q[:, 2].tolist()},
            "Q_orientation_average": {"Qext": q_avg[:, 0].tolist(), "Qabs": q_avg[:, 1].tolist(),
                                      "Qsca": q_avg[:, 2].tolist(), "per": "incident polarization"},
            "warm_start": warm_report,
            "e2e": {"value": e2e_value, "unit": "matvecs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "clocks": clk,
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

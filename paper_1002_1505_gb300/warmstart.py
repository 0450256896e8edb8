"""Learned warm start for the DDA solve: data from the solver, training, use.

The solver (dda_solve) accepts any initial guess.  This module trains the
library's 3-D U-Net (dda_unet_*) to predict the local field E_loc = alpha^{-1} P
from per-voxel features of a target (occupancy, permittivity, incident field)
and turns its prediction into a guess P0 = alpha E_loc.  The network learns
the correction E_loc - E_inc: for a small sphere in the static limit the
Lorentz local field equals the incident field, so the network-free guess
alpha E_inc is its starting point.  Every step runs in
the library: solutions come from dda_solve, features/targets/guesses from
dda_unet_features / dda_unet_targets / dda_unet_warm_start, training from
dda_unet_loss_grad and dda_unet_adamw.  torch only holds device buffers and
gathers mini-batches.

Random problems: spheres, ellipsoids and hexagonal prisms on boxes up to
max_box^3, Re m in [1.1, 2.5], Im m in [0, 0.5], x in [1, 10], one uniform
orientation (workloads.random_unet_sample); kd is capped at 0.8/|m| so that
every problem stays in the DDA's range of validity (|m| kd < 1).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

from . import dda as D
from . import workloads as W

CIN, COUT = 9, 6
DEFAULT_CH = (12, 24, 32, 48)


def grid_dims(box, mult: int = 8) -> Tuple[int, int, int]:
    return tuple(int(math.ceil(b / mult) * mult) for b in box)


def problem(index: int, max_box: int, device: int = 0, stream=None):
    """Context for random problem `index` (target, incidence, Green tensor, alpha)."""
    shape, shpar, m, x, ori = W.random_unet_sample(index, max_box)
    ctx = D.Context(device, stream)
    n, box = ctx.dda_setup_shape(shape, shpar)
    kd = min(ctx.dda_kd_from_x(x)[0], 0.8 / abs(m))
    ctx.dda_set_incident(kd, [ori], [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("GKDLDR", m)
    return ctx


def generate(indices, max_box: int, grid, device: int = 0, group: int = 8, tol: float = 1e-5, keep: bool = False):
    """Solve the random problems `indices` and return device tensors (X, T, M) on the fixed grid.

    Each problem gives two samples (its two polarizations).  Problems are solved
    `group` at a time with dda_solve_batch.  keep=True also returns the
    contexts (for the residual loss), else they are closed.
    """
    import torch
    V = grid[0] * grid[1] * grid[2]
    S = 2 * len(indices)
    X = torch.zeros((S, grid[2], grid[1], grid[0], CIN), dtype=torch.float32, device="cuda")
    T = torch.zeros((S, grid[2], grid[1], grid[0], COUT), dtype=torch.float32, device="cuda")
    M = torch.zeros((S, grid[2], grid[1], grid[0]), dtype=torch.float32, device="cuda")
    iters, kept = [], []
    for g0 in range(0, len(indices), group):
        ctxs = [problem(i, max_box, device) for i in indices[g0:g0 + group]]
        ps = [torch.zeros((c.nrhs, 3, c.n), dtype=torch.complex128, device="cuda") for c in ctxs]
        reps, sts, overall = D.dda_solve_batch(ctxs, ps, precision="MIXED", tol=tol, maxit=3000)
        for k, (c, p, r) in enumerate(zip(ctxs, ps, reps)):
            s = 2 * (g0 + k)
            D.dda_unet_features(c, X[s:s + 2], grid)
            D.dda_unet_targets(c, p, T[s:s + 2], M[s:s + 2], grid, residual=True)
            iters.extend(x["iters"] for x in r)
        torch.cuda.synchronize()
        if keep:
            kept.extend(ctxs)
        else:
            for c in ctxs:
                c.close()
    return (X, T, M, iters, kept) if keep else (X, T, M, iters)


def train(net: "D.UNet", X, T, M, grid, steps: int, batch: int, lr: float = 2e-3, seed: int = 0,
          wd: float = 0.0) -> List[float]:
    """AdamW on random mini-batches; cosine learning-rate decay. Returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    S = X.shape[0]
    hist = []
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(S, size=min(batch, S), replace=False)).cuda()
        xb, tb, mb = X[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous()
        loss = net.dda_unet_loss_grad(xb, tb, mb, grid)
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps)))
        net.dda_unet_adamw(rate, wd=wd)
        hist.append(loss)
    return hist


def zero_head(net: "D.UNet"):
    """Zero the 1x1x1 output layer: the untrained network then predicts no
    correction, i.e. its guess starts as the alpha E_inc guess."""
    theta = net.dda_unet_get_params(0)
    c1 = net.ch[0]
    theta[-(c1 * COUT + COUT):] = 0.0
    net.dda_unet_set_params(theta)


def train_residual(net: "D.UNet", ctxs, X, T, M, grid, steps: int, per_step: int = 8, lr: float = 1e-3,
                   res_weight: float = 1.0, mse_weight: float = 1.0, seed: int = 0,
                   wd: float = 0.0) -> List[Tuple[float, float]]:
    """Train on mse_weight * MSE(E_loc) + res_weight * mean |E - A P0|^2/|E|^2 over `per_step` problems per step.

    The residual term goes through the library's own product and its adjoint
    (dda_unet_residual_grad), so the network is trained on the quantity the
    Krylov solver starts from.  Returns (mse, residual) per step."""
    import torch
    rng = np.random.default_rng(seed)
    K = len(ctxs)
    hist = []
    for it in range(steps):
        pick = rng.choice(K, size=min(per_step, K), replace=False)
        idx = torch.from_numpy(np.stack([2 * pick, 2 * pick + 1], axis=1).reshape(-1)).cuda()
        xb, tb, mb = X[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous()
        y = torch.empty_like(tb)
        gy = torch.empty_like(tb)
        net.dda_unet_forward_train(xb, y, grid)
        mse = net.dda_unet_mse(y, tb, mb, gy, grid, weight=mse_weight)
        res = 0.0
        for k, ci in enumerate(pick):
            res += D.dda_unet_residual_grad(ctxs[ci], y[2 * k:2 * k + 2], gy[2 * k:2 * k + 2], grid,
                                            weight=res_weight / (2 * len(pick)))
        net.dda_unet_backward(gy, grid)
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps)))
        net.dda_unet_adamw(rate, wd=wd)
        hist.append((mse / mse_weight if mse_weight else 0.0, res / res_weight if res_weight else 0.0))
    return hist


def residual_of_guess(ctxs, grid, ys=None) -> float:
    """Mean |E - A P0|^2/|E|^2 over the contexts' right-hand sides for outputs ys (None: y = 0, the alpha E_inc guess)."""
    import torch
    tot, cnt = 0.0, 0
    for k, c in enumerate(ctxs):
        y = torch.zeros((c.nrhs, grid[2], grid[1], grid[0], COUT), dtype=torch.float32, device="cuda") if ys is None else ys[k]
        gy = torch.zeros_like(y)
        tot += D.dda_unet_residual_grad(c, y, gy, grid)
        cnt += c.nrhs
    return tot / cnt


def warm_guess(ctx: "D.Context", net: "D.UNet", grid=None, chunk: int = 0):
    """Initial guess P0 (complex128 [nrhs, 3, N]) for a context from the network (forward pass in
    chunks of `chunk` right-hand sides when > 0, to bound the activations of large grids)."""
    import torch
    grid = grid_dims(ctx.box) if grid is None else grid
    x = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0], CIN), dtype=torch.float32, device="cuda")
    y = torch.empty((ctx.nrhs, grid[2], grid[1], grid[0], COUT), dtype=torch.float32, device="cuda")
    D.dda_unet_features(ctx, x, grid)
    step = chunk if chunk > 0 else ctx.nrhs
    for b0 in range(0, ctx.nrhs, step):
        net.dda_unet_forward(x[b0:b0 + step].contiguous(), y[b0:b0 + step], grid)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    D.dda_unet_warm_start(ctx, y, grid, p, residual=True)
    net.dda_unet_check_fault()
    return p


def local_field_guess(ctx: "D.Context", grid=None):
    """The network-free guess P0 = alpha E_inc (the local field taken as the incident field)."""
    import torch
    grid = grid_dims(ctx.box) if grid is None else grid
    x = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0], CIN), dtype=torch.float32, device="cuda")
    D.dda_unet_features(ctx, x, grid)
    y = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0], COUT), dtype=torch.float32, device="cuda")
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    D.dda_unet_warm_start(ctx, y, grid, p, residual=True)  # zero correction: E_loc = E_inc
    return p


def train_quick(problems: int, steps: int, max_box: int = 16, widths=(16, 32, 48, 64), seed: int = 5):
    """A network trained from scratch on `problems` random problems (two solutions each) for `steps`
    AdamW steps of 16 samples, output layer zeroed at start (the recipe of main(), smaller)."""
    grid = (max_box, max_box, max_box)
    X, T, M, _ = generate(list(range(problems)), max_box, grid)
    net = D.UNet(0, None, CIN, COUT, tuple(widths), seed=seed)
    zero_head(net)
    train(net, X, T, M, grid, steps=steps, batch=16, lr=1e-3)
    del X, T, M
    return net


def evaluate(net: "D.UNet", indices, max_box: int, grid=None, tol: float = 1e-5, maxit: int = 3000):
    """Iterations to tol (true residual) from a cold start, the alpha E_inc guess and the network guess:
    per problem and start, (iterations, largest true residual, right-hand sides left above tol after
    maxit iterations)."""
    import torch
    rows = []
    for i in indices:
        ctx = problem(i, max_box)
        out = {}
        for name in ("cold", "alpha_einc", "network"):
            if name == "cold":
                p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
                warm = False
            elif name == "alpha_einc":
                p, warm = local_field_guess(ctx, grid), True
            else:
                p, warm = warm_guess(ctx, net, grid), True
            reps, _ = ctx.dda_solve(p, precision="MIXED", tol=tol, maxit=maxit, warm_start=warm,
                                    raise_on_noconv=False)
            out[name] = (sum(r["iters"] for r in reps), max(r["true_rel_resid"] for r in reps),
                         sum(1 for r in reps if r["true_rel_resid"] > tol))
        rows.append(out)
        ctx.close()
    return rows


def main():
    """Config-4-style evaluation: train on solver output, compare iterations to 1e-5 on held-out problems
    (cold start, alpha E_inc, network) and, with --large, on the 160 x 128 hexagonal prism."""
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-problems", type=int, default=8192)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--max-box", type=int, default=16)
    ap.add_argument("--heldout", type=int, default=32)
    ap.add_argument("--large", action="store_true")
    args = ap.parse_args()
    grid = (args.max_box, args.max_box, args.max_box)
    t0 = time.time()
    X, T, M, _ = generate(list(range(args.train_problems)), args.max_box, grid)
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    m = M[..., None]
    mse0 = float((m * T * T).sum() / (m.sum() * COUT))
    net = D.UNet(0, None, CIN, COUT, (16, 32, 48, 64), seed=5)
    zero_head(net)
    t0 = time.time()
    hist = train(net, X, T, M, grid, steps=args.steps, batch=16, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del X, T, M
    torch.cuda.empty_cache()  # the training set's memory back to the device for the library's own buffers
    rows = evaluate(net, list(range(100000, 100000 + args.heldout)), args.max_box, grid)
    out = {"train_samples": 2 * args.train_problems, "max_box": args.max_box, "steps": args.steps,
           "params": int(net.nparams),
           "generate_s": round(t_gen, 1), "train_s": round(t_train, 1),
           "mse_no_network": mse0, "mse_final": float(np.mean(hist[-200:])),
           "heldout_problems": args.heldout,
           "heldout_iterations": {k: int(sum(r[k][0] for r in rows)) for k in ("cold", "alpha_einc", "network")},
           "heldout_max_resid": {k: float(max(r[k][1] for r in rows)) for k in ("cold", "alpha_einc", "network")},
           "heldout_unconverged_rhs": {k: int(sum(r[k][2] for r in rows)) for k in ("cold", "alpha_einc", "network")}}
    print(json.dumps(out), flush=True)  # the held-out result first; --large adds a second line
    if args.large:
        w = W.HEXPRISM160
        ctx = D.Context(0)
        D.setup_workload(ctx, w)
        big = grid_dims(ctx.box)
        # autotune the product schedules before any timed solve
        D.dda_profile_matvec(ctx, ctx.nrhs, D.DDA_C64, 1)
        D.dda_profile_matvec(ctx, ctx.nrhs, D.DDA_C128, 1)
        res = {}
        for name in ("cold", "alpha_einc", "network"):
            torch.cuda.synchronize()
            t0 = time.time()
            if name == "cold":
                p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
                warm = False
            elif name == "alpha_einc":
                p, warm = local_field_guess(ctx, big), True
            else:
                p, warm = warm_guess(ctx, net, big, chunk=2), True
            torch.cuda.synchronize()
            t_guess = time.time() - t0
            t0 = time.time()
            reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000, warm_start=warm,
                                    raise_on_noconv=False)
            torch.cuda.synchronize()
            res[name] = {"iterations": int(sum(r["iters"] for r in reps)), "solve_s": round(time.time() - t0, 3),
                         "guess_s": round(t_guess, 3), "max_resid": float(max(r["true_rel_resid"] for r in reps))}
            del p
        out["hexprism160"] = {"grid": list(big), "nrhs": ctx.nrhs, **res}
        ctx.close()
        print(json.dumps(out))


if __name__ == "__main__":
    main()

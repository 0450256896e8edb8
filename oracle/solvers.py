"""Linear solvers for A P = E (guide, "Choice of Iterative Algorithm").

* lu_solve: dense LU with partial pivoting (numpy/LAPACK) for tiny targets.
* bicgstab: the stabilized bi-conjugate gradient of van der Vorst (1992), the
  method behind the guide's PBCGST option, unpreconditioned, initial shadow
  residual equal to the initial residual.
* ccg: the complex conjugate gradient of Petravic & Kuo-Petravic (1979) (the
  guide's PETRKP): conjugate gradients on the normal equations
  A^H A P = A^H E, two products per iteration.  Because A is complex
  symmetric, A^H x = conj(A conj(x)).
* bicgstab_l: BiCGstab(l) of Sleijpen & Fokkema (1993), the family behind the
  guide's PBCGS2 option (l = 2; the guide's routine adds Sleijpen & van der
  Vorst's reliability refinements, which are not reproduced): each cycle runs
  l BiCG steps, then a minimal-residual polynomial of degree l (modified
  Gram-Schmidt form).  With l = 1 it is BiCGstab.

All iterate in FP64 and stop on the true relative residual |E - A P| / |E|;
`normal_eq_ratio` evaluates the guide's own stopping quantity
|A^H A P - A^H E| / |A^H E| (guide, eq. err_tol) for reporting.
"""
from __future__ import annotations

import numpy as np


def lu_solve(a: np.ndarray, e: np.ndarray) -> np.ndarray:
    return np.linalg.solve(a, e)


def _dot(u, v):
    return np.vdot(u, v)  # conj(u) . v


def bicgstab(apply_a, e: np.ndarray, x0=None, tol: float = 1e-10, maxit: int = 2000):
    """Returns (x, iterations, relative residual history)."""
    x = np.zeros_like(e) if x0 is None else x0.astype(np.complex128).copy()
    r = e - apply_a(x) if x0 is not None else e.copy()
    norm_e = np.linalg.norm(e)
    hist = [np.linalg.norm(r) / norm_e]
    if hist[-1] <= tol:
        return x, 0, hist
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(e)
    p = np.zeros_like(e)
    for it in range(1, maxit + 1):
        rho = _dot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_a(p)
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) / norm_e <= tol:
            x = x + alpha * p
            hist.append(np.linalg.norm(s) / norm_e)
            return x, it, hist
        t = apply_a(s)
        omega = _dot(t, s) / _dot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        hist.append(np.linalg.norm(r) / norm_e)
        if hist[-1] <= tol:
            return x, it, hist
        rho_old = rho
    return x, maxit, hist


def ccg(apply_a, e: np.ndarray, x0=None, tol: float = 1e-10, maxit: int = 5000):
    """CG on the normal equations (CGNR). Returns (x, iterations, relative residual history)."""
    def apply_ah(v):
        return np.conj(apply_a(np.conj(v)))

    x = np.zeros_like(e) if x0 is None else x0.astype(np.complex128).copy()
    r = e - apply_a(x) if x0 is not None else e.copy()
    norm_e = np.linalg.norm(e)
    hist = [np.linalg.norm(r) / norm_e]
    if hist[-1] <= tol:
        return x, 0, hist
    z = apply_ah(r)
    p = z.copy()
    zz = np.real(_dot(z, z))
    for it in range(1, maxit + 1):
        w = apply_a(p)
        alpha = zz / np.real(_dot(w, w))
        x = x + alpha * p
        r = r - alpha * w
        hist.append(np.linalg.norm(r) / norm_e)
        if hist[-1] <= tol:
            return x, it, hist
        z = apply_ah(r)
        zz_new = np.real(_dot(z, z))
        p = z + (zz_new / zz) * p
        zz = zz_new
    return x, maxit, hist


def bicgstab_l(apply_a, e: np.ndarray, ell: int = 2, x0=None, tol: float = 1e-10, maxit: int = 2000):
    """BiCGstab(l).  Returns (x, iterations, relative residual history); one "iteration" is one BiCG
    step (two products, as for bicgstab), so a cycle counts l iterations; the residual is checked at
    the end of every cycle."""
    x = np.zeros_like(e) if x0 is None else x0.astype(np.complex128).copy()
    r0 = e - apply_a(x) if x0 is not None else e.copy()
    norm_e = np.linalg.norm(e)
    hist = [np.linalg.norm(r0) / norm_e]
    if hist[-1] <= tol:
        return x, 0, hist
    rt = r0.copy()                      # shadow residual
    u = [np.zeros_like(e) for _ in range(ell + 1)]
    r = [r0] + [None] * ell
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    it = 0
    while it < maxit:
        rho0 = -omega * rho0
        # BiCG part: r[0..j+1] and u[0..j+1] span the Krylov directions of this cycle
        for j in range(ell):
            rho1 = _dot(rt, r[j])
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = apply_a(u[j])
            alpha = rho0 / _dot(rt, u[j + 1])
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = apply_a(r[j])
            x = x + alpha * u[0]
        it += ell
        # MR part: minimise |r0 - sum_j gamma_j r_j| (modified Gram-Schmidt on r_1..r_l)
        tau = np.zeros((ell + 1, ell + 1), dtype=np.complex128)
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1, dtype=np.complex128)
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = _dot(r[i], r[j]) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sigma[j] = np.real(_dot(r[j], r[j]))
            gp[j] = _dot(r[j], r[0]) / sigma[j]
        g = np.zeros(ell + 1, dtype=np.complex128)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1, dtype=np.complex128)
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * r[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            x = x + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        hist.append(np.linalg.norm(r[0]) / norm_e)
        if hist[-1] <= tol:
            return x, it, hist
        if omega == 0 or rho0 == 0:
            break
    return x, it, hist


def normal_eq_ratio(apply_a, x, e) -> float:
    def apply_ah(v):
        return np.conj(apply_a(np.conj(v)))
    r = apply_a(x) - e
    return float(np.linalg.norm(apply_ah(r)) / np.linalg.norm(apply_ah(e)))

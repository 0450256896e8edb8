"""Linear solvers for A P = E (guide, "Choice of Iterative Algorithm").

* lu_solve: dense LU with partial pivoting (numpy/LAPACK) for tiny targets.
* bicgstab: the stabilized bi-conjugate gradient of van der Vorst (1992), the
  method behind the guide's PBCGST option, unpreconditioned, initial shadow
  residual equal to the initial residual.
* ccg: the complex conjugate gradient of Petravic & Kuo-Petravic (1979) (the
  guide's PETRKP): conjugate gradients on the normal equations
  A^H A P = A^H E, two products per iteration.  Because A is complex
  symmetric, A^H x = conj(A conj(x)).

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


def normal_eq_ratio(apply_a, x, e) -> float:
    def apply_ah(v):
        return np.conj(apply_a(np.conj(v)))
    r = apply_a(x) - e
    return float(np.linalg.norm(apply_ah(r)) / np.linalg.norm(apply_ah(e)))

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
* cocg: conjugate orthogonal conjugate gradients (van der Vorst & Melissen
  1990): CG with the unconjugated bilinear form x^T y, valid because A is
  complex symmetric (A^T = A); one product per iteration.
* qmr_cs: quasi-minimal residual for complex symmetric systems (Freund 1992),
  the guide's QMRCCG family: the complex-symmetric Lanczos process (basis
  vectors orthogonal in x^T y, scaled to unit 2-norm) and, at each step, the
  least-squares problem min |rho_1 e_1 - H_n z| of its tridiagonal
  (n+1) x n matrix solved by complex Givens rotations; one product per
  iteration.

All iterate in FP64 and stop on the true relative residual |E - A P| / |E|;
`normal_eq_ratio` evaluates the guide's own stopping quantity
|A^H A P - A^H E| / |A^H E| (guide, eq. err_tol) for reporting.

TEST INFRASTRUCTURE ONLY (see the package docstring).
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


def cocg(apply_a, e: np.ndarray, x0=None, tol: float = 1e-10, maxit: int = 5000):
    """COCG (van der Vorst & Melissen 1990).  Returns (x, iterations, relative residual history)."""
    x = np.zeros_like(e) if x0 is None else x0.astype(np.complex128).copy()
    r = e - apply_a(x) if x0 is not None else e.copy()
    norm_e = np.linalg.norm(e)
    hist = [np.linalg.norm(r) / norm_e]
    if hist[-1] <= tol:
        return x, 0, hist
    p = r.copy()
    rho = np.sum(r * r)  # r^T r, no conjugation
    it = 0
    for it in range(1, maxit + 1):
        q = apply_a(p)
        mu = np.sum(p * q)
        if mu == 0 or rho == 0:
            break
        alpha = rho / mu
        x = x + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r) / norm_e)
        if hist[-1] <= tol:
            break
        rho_new = np.sum(r * r)
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, it, hist


def _givens(a: complex, b: complex):
    """Complex rotation [[c, s], [-conj(s), c]] (c real) taking (a, b) to (r, 0); returns (c, s, r)."""
    if b == 0:
        return 1.0, 0j, a
    if a == 0:
        return 0.0, 1.0 + 0j, b
    h = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    return abs(a) / h, ph * np.conj(b) / h, ph * h


def qmr_cs(apply_a, e: np.ndarray, x0=None, tol: float = 1e-10, maxit: int = 5000):
    """QMR for complex symmetric A (Freund 1992), without look-ahead.

    Returns (x, iterations, relative residual history, quasi-residual history); the quasi-residual
    |tau_{n+1}| / |E| bounds the true relative residual from below by 1/sqrt(n+1) (unit 2-norm basis).
    The stopping test uses the true residual E - A x (an extra product, the oracle does not count it).
    """
    x = np.zeros_like(e) if x0 is None else x0.astype(np.complex128).copy()
    r0 = e - apply_a(x) if x0 is not None else e.copy()
    norm_e = np.linalg.norm(e)
    hist = [np.linalg.norm(r0) / norm_e]
    qhist = [hist[0]]
    if hist[-1] <= tol:
        return x, 0, hist, qhist
    rho = np.linalg.norm(r0)          # rho_1
    v = r0 / rho                      # v_1
    v_prev = np.zeros_like(e)
    delta_prev = 1.0 + 0j
    rho_n = rho                       # rho_n (scale of v_n)
    tau_bar = rho + 0j                # rotated right-hand side entry
    d_prev = np.zeros_like(e)         # d_{n-1}
    d_prev2 = np.zeros_like(e)        # d_{n-2}
    c1, s1 = 1.0, 0j                  # G_{n-1}
    c2, s2 = 1.0, 0j                  # G_{n-2}
    it = 0
    for it in range(1, maxit + 1):
        delta = np.sum(v * v)         # v_n^T v_n
        if delta == 0:
            break                     # Lanczos breakdown (no look-ahead)
        av = apply_a(v)
        alpha = np.sum(v * av) / delta
        beta = rho_n * delta / delta_prev if it > 1 else 0j
        w = av - alpha * v - beta * v_prev
        rho_next = np.linalg.norm(w)
        # column n of H: beta at row n-1, alpha at row n, rho_next at row n+1
        r_nm2 = s2 * beta                       # G_{n-2} on (0, beta)
        f = c2 * beta
        r_nm1 = c1 * f + s1 * alpha             # G_{n-1} on (f, alpha)
        g = -np.conj(s1) * f + c1 * alpha
        c, s, r_nn = _givens(g, rho_next)       # G_n on (g, rho_next)
        if r_nn == 0:
            break
        d = (v - r_nm1 * d_prev - r_nm2 * d_prev2) / r_nn
        tau = c * tau_bar
        tau_bar = -np.conj(s) * tau_bar
        x = x + tau * d
        hist.append(np.linalg.norm(e - apply_a(x)) / norm_e)
        qhist.append(abs(tau_bar) / norm_e)
        if hist[-1] <= tol or rho_next == 0:
            break
        d_prev2, d_prev = d_prev, d
        c2, s2, c1, s1 = c1, s1, c, s
        v_prev, v = v, w / rho_next
        delta_prev, rho_n = delta, rho_next
    return x, it, hist, qhist


def normal_eq_ratio(apply_a, x, e) -> float:
    def apply_ah(v):
        return np.conj(apply_a(np.conj(v)))
    r = apply_a(x) - e
    return float(np.linalg.norm(apply_ah(r)) / np.linalg.norm(apply_ah(e)))

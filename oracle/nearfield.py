"""Electric and magnetic fields in or near the target from a solved P (guide, "Postprocessing:
Calculating E and B In or Near the Target" -- the DDfield program).

TEST INFRASTRUCTURE ONLY (see the package docstring).

At a point r (Target Frame, lattice units), time factor exp(-i w t), Gaussian units, |E0| = 1:
    E(r) = E_inc(r) + sum_j phi(|r - r_j|) E_dip(r - r_j; P_j)
    B(r) = B_inc(r) + sum_j phi(|r - r_j|) B_dip(r - r_j; P_j)
with the incident plane wave E_inc = e exp(i k.r), B_inc = khat x E_inc, and the retarded fields of
an oscillating point dipole p at distance R = R n (Jackson, Classical Electrodynamics, eqs. 9.18 and
9.19, Gaussian form):
    E_dip = exp(i k R) { k^2 (n x p) x n / R + [3 n (n.p) - p] (1/R^3 - i k / R^2) }
    B_dip = exp(i k R) k^2 (n x p) (1/R) (1 - 1/(i k R)).
The guide suppresses the divergent contribution of dipoles closer than one lattice spacing d with a
factor phi(R) that vanishes faster than R^3 and leaves the field of every dipole at R >= d
untouched; its form is delegated to Draine & Flatau (2008).  Reading taken here:
    phi(R) = (R/d)^4 (5 - 4 R/d) for R < d, 1 otherwise
(continuous with a continuous first derivative at R = d, ~ R^4 as R -> 0).
"""
from __future__ import annotations

import numpy as np


def suppression(R):
    """phi(R) in lattice units (d = 1)."""
    R = np.asarray(R, dtype=np.float64)
    return np.where(R < 1.0, R ** 4 * (5.0 - 4.0 * R), 1.0)


def dipole_fields(rvec, p, k):
    """E and B at separations rvec (M, 3) (all nonzero) of point dipoles p (M, 3)."""
    R = np.linalg.norm(rvec, axis=-1)
    n = rvec / R[:, None]
    ph = np.exp(1j * k * R)
    nxp = np.cross(n, p)
    ndp = np.sum(n * p, axis=-1)
    E = ph[:, None] * (k * k * np.cross(nxp, n) / R[:, None]
                       + (3 * n * ndp[:, None] - p) * (1 / R ** 3 - 1j * k / R ** 2)[:, None])
    B = ph[:, None] * k * k * nxp / R[:, None] * (1 - 1 / (1j * k * R))[:, None]
    return E, B


def fields_at(points, kd, r, p, k_tf, e_tf, periods=None, gamma=0.0):
    """Total E and B (each (M, 3) complex) at points (M, 3) for one RHS: sites r (N, 3), solution p
    (3, N), incident wave vector k_tf (3,) and polarization e_tf (3,) in the TF.

    Periodic targets (periods = (P_y, P_z), a zero for an axis without repetition): the replica of
    the unit cell displaced by R carries P exp(i k.R), and each dipole's contribution is multiplied by
    the same cutoff exp[-(gamma k D)^4] of its distance D to the point as the periodic interaction
    (oracle.periodic), replicas dropped where (gamma k D)^4 > 40: the guide's DDfield lets phi(r)
    suppress the distant dipoles of an infinite target so that the sums can be truncated; the near
    suppression below one lattice spacing stays as for a finite target."""
    k = float(kd)
    khat = np.asarray(k_tf, float) / np.linalg.norm(k_tf)
    pts = np.asarray(points, dtype=np.float64)
    Eo = np.zeros((len(pts), 3), dtype=np.complex128)
    Bo = np.zeros((len(pts), 3), dtype=np.complex128)
    pt = p.T
    periodic = periods is not None and (periods[0] > 0 or periods[1] > 0)
    if periodic:
        from . import periodic as per
        ext = float(np.max(np.linalg.norm(pts[:, None, 1:] - r[None, :, 1:], axis=-1)))
        reps = per.replica_offsets(periods, k, gamma, extra=ext)
        bloch = np.exp(1j * (reps @ np.asarray(k_tf, float)))
    else:
        reps = np.zeros((1, 3))
        bloch = np.ones(1, dtype=np.complex128)
    # every (replica, site) pair as one flat list: separation, moment with its Bloch phase
    pm = (bloch[:, None, None] * pt[None, :, :]).reshape(-1, 3)
    for i, x in enumerate(pts):
        einc = np.asarray(e_tf) * np.exp(1j * np.dot(k_tf, x))
        d = (x[None, None, :] - r[None, :, :] - reps[:, None, :]).reshape(-1, 3)
        D = np.linalg.norm(d, axis=-1)
        keep = D > 0
        if periodic:
            keep &= (gamma * k * D) ** 4 <= per.CUTOFF_EXP
        E, B = dipole_fields(d[keep], pm[keep], k)
        w = suppression(D[keep])
        if periodic:
            w = w * np.exp(-(gamma * k * D[keep]) ** 4)
        Eo[i] = einc + np.sum(w[:, None] * E, axis=0)
        Bo[i] = np.cross(khat, einc) + np.sum(w[:, None] * B, axis=0)
    return Eo, Bo

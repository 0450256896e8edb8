"""Target orientation and incident beam, restated from the guide.

* "Orientation of the Target in the Lab Frame": a1, a2, a3 in the LF from
  (Theta, Phi, beta), and the inverse relations giving x_LF, y_LF, z_LF in terms
  of a1, a2, a3.  Because the target axes are known in the Target Frame, the
  inverse relations give the Lab-Frame unit vectors in the TF directly.
* "Incident Polarization State": k along x_LF, e01 user given (normalized),
  e02 = x_LF x e01*.
* "Scattering directions" (CMDFRM = LFRAME): n_s = x cos(th) + y sin(th) cos(ph)
  + z sin(th) sin(ph); the scattered basis is theta_hat, phi_hat of that
  direction ("Scattering Amplitude Matrix" section).
* "Sampling in Theta, Phi, and beta" / "Orientational Averaging": beta and
  Phi at the midpoints of NBETA / NPHI equal intervals, uniform weights;
  cos(Theta) uniform: NTHETA odd -> the end points included and Simpson
  weights, NTHETA even -> interval midpoints and equal weights.  The guide
  writes the odd-NTHETA weights as (1/3, 4/3, 2/3)/(NTHETA NPHI), which would
  not sum to one; they are taken here as Simpson's rule on NTHETA - 1
  intervals of cos(Theta), i.e. (1/3, 4/3, 2/3, ..., 4/3, 1/3)/(NTHETA - 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def lab_axes_in_tf(beta: float, theta: float, phi: float, a1_tf, a2_tf):
    """Return x_LF, y_LF, z_LF expressed in Target-Frame components."""
    a1 = np.asarray(a1_tf, float)
    a2 = np.asarray(a2_tf, float)
    a3 = np.cross(a1, a2)
    ct, st = np.cos(theta), np.sin(theta)
    cb, sb = np.cos(beta), np.sin(beta)
    cp, sp = np.cos(phi), np.sin(phi)
    x_lf = a1 * ct - a2 * st * cb + a3 * st * sb
    y_lf = a1 * st * cp + a2 * (ct * cb * cp - sb * sp) - a3 * (ct * sb * cp + cb * sp)
    z_lf = a1 * st * sp + a2 * (ct * cb * sp + sb * cp) - a3 * (ct * sb * sp - cb * cp)
    return x_lf, y_lf, z_lf


def target_axes_in_lf(beta: float, theta: float, phi: float):
    """a1, a2, a3 in Lab-Frame components (the forward relations)."""
    ct, st = np.cos(theta), np.sin(theta)
    cb, sb = np.cos(beta), np.sin(beta)
    cp, sp = np.cos(phi), np.sin(phi)
    a1 = np.array([ct, st * cp, st * sp])
    a2 = np.array([-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp])
    a3 = np.array([st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)])
    return a1, a2, a3


def polarizations_lf(e01_lf, iorth: int = 2):
    """Normalized e01 and, for IORTH=2, e02 = x_LF x e01* (Lab-Frame complex 3-vectors)."""
    e01 = np.asarray(e01_lf, dtype=np.complex128)
    e01 = e01 / np.sqrt(np.sum(np.abs(e01) ** 2))
    out = [e01]
    if iorth == 2:
        out.append(np.cross(np.array([1.0, 0.0, 0.0]), np.conj(e01)))
    return out


def lf_to_tf(v_lf, axes):
    """Lab-Frame components -> Target-Frame components (axes = x_LF, y_LF, z_LF in TF)."""
    x, y, z = axes
    v = np.asarray(v_lf)
    return v[0] * x + v[1] * y + v[2] * z


def incidence(kd: float, ori, a1_tf, a2_tf, e01_lf, iorth: int = 2):
    """For one orientation: k vector and incident polarizations, all in TF components."""
    beta, theta, phi = ori
    axes = lab_axes_in_tf(beta, theta, phi, a1_tf, a2_tf)
    k_tf = kd * axes[0]
    pols_lf = polarizations_lf(e01_lf, iorth)
    pols_tf = [lf_to_tf(e, axes) for e in pols_lf]
    return k_tf, pols_tf, pols_lf, axes


def scattering_basis_lf(theta_s: float, phi_s: float):
    """n_s, theta_hat_s, phi_hat_s in Lab-Frame components (LFRAME convention)."""
    ct, st = np.cos(theta_s), np.sin(theta_s)
    cp, sp = np.cos(phi_s), np.sin(phi_s)
    n = np.array([ct, st * cp, st * sp])
    th = np.array([-st, ct * cp, ct * sp])
    ph = np.array([0.0, -sp, cp])
    return n, th, ph


def orientation_grid(beta_deg, nbeta: int, theta_deg, ntheta: int, phi_deg, nphi: int):
    """(orientations [(beta, Theta, Phi)] in radians, weights summing to one); Phi varies fastest,
    then Theta, then beta.  *_deg = (min, max) in degrees."""
    def mids(lo, hi, n):
        return [lo + (hi - lo) * (i + 0.5) / n for i in range(n)]
    betas = mids(beta_deg[0], beta_deg[1], nbeta)
    phis = mids(phi_deg[0], phi_deg[1], nphi)
    c0, c1 = np.cos(np.radians(theta_deg[0])), np.cos(np.radians(theta_deg[1]))
    if ntheta % 2 == 1:
        if ntheta == 1:
            cosv, wt = [c0], [1.0]
        else:
            cosv = [c0 + (c1 - c0) * i / (ntheta - 1) for i in range(ntheta)]
            wt = [(1.0 if i in (0, ntheta - 1) else (4.0 if i % 2 == 1 else 2.0)) / 3.0 / (ntheta - 1)
                  for i in range(ntheta)]
    else:
        cosv = [c0 + (c1 - c0) * (i + 0.5) / ntheta for i in range(ntheta)]
        wt = [1.0 / ntheta] * ntheta
    oris, w = [], []
    for b in betas:
        for t, wth in zip(cosv, wt):
            for f in phis:
                oris.append((np.radians(b), float(np.arccos(np.clip(t, -1.0, 1.0))), np.radians(f)))
                w.append(wth / (nbeta * nphi))
    return oris, np.array(w)


def dielectric_axes(theta_df: float, phi_df: float, beta_df: float):
    """Principal axes e_1, e_2, e_3 of a site's dielectric tensor in Target-Frame components (guide,
    "Composite Targets with Anisotropic Constituents": rotate by theta_DF about y_TF, then phi_DF
    about x_TF, then beta_DF about e_1)."""
    ct, st = np.cos(theta_df), np.sin(theta_df)
    cp, sp = np.cos(phi_df), np.sin(phi_df)
    cb, sb = np.cos(beta_df), np.sin(beta_df)
    e1 = np.array([ct, st * cp, st * sp])
    e2 = np.array([-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp])
    e3 = np.array([st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)])
    return e1, e2, e3

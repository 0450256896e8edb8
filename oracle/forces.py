"""Radiative force and torque on the dipole array (guide, "Calculation of <cos theta>, Radiative
Force, and Radiation Torque").

TEST INFRASTRUCTURE ONLY (see the package docstring).

The guide defines the efficiency vectors
    Q_pr    = F_rad / (pi a_eff^2 u_rad),    Q_Gamma = k Gamma_rad / (pi a_eff^2 u_rad),
with u_rad = |E0|^2 / 8 pi (here |E0| = 1), writes Q_pr = Q_ext khat - Q_sca g with
g = (1/C_sca) int dOmega (dC_sca/dOmega) n, reports both vectors in the Target Frame, and delegates
the torque formulas to Draine & Weingartner (1996).  Restated here from the time-averaged force and
torque on point dipoles (fields Re[E exp(-i w t)]):
    torque on dipole j about the reference point:  1/2 Re(P_j x E_j^*) + r_j x F_j,
    force on dipole j:                              F_j = 1/2 Re sum_a P_ja grad E_ja^*,
where E_j is the field at site j from every source but the dipole's own static self-field.

Incident part (E_inc = e exp(i k.r), grad E_inc^* = -i k E_inc^*):
    Gamma_ext = sum_j [ 1/2 Re(P_j x E_inc,j^*) + (k/2) Im(P_j . E_inc,j^*) r_j x khat ].
Part from the array's own field.  Split the dipole field tensor G(R) (E = G(R) p) into its real and
imaginary parts; the real part is the time-symmetric interaction, whose forces and torques cancel
over the closed array; the imaginary part is smooth, equals (2/3) k^3 I at R = 0 (the radiation
reaction of each dipole on itself) and is the plane-wave integral
    Im G(R) = (k^3 / 4 pi) oint dOmega (I - n n) exp(i k n . R).
Inserting it gives, with g(n) = sum_j P_j exp(-i k n.r_j), f = g - n (n.g),
T(n) = sum_j r_j P_j^T exp(-i k n.r_j) and h(n) = T(n) f(n)^*:
    Gamma_self = (k^3 / 8 pi) oint dOmega Im[g x f^*] - (k^4 / 8 pi) oint dOmega Re[h] x n,
    F_self     = -(k^4 / 8 pi) oint dOmega |f|^2 n      (= -u_rad C_sca g).
Those far-field forms are what the CUDA library evaluates; `direct_force_torque` below evaluates the
same physical quantities site by site with the full (real and imaginary) tensor and its gradient,
which pins both the split and the plane-wave identity.  Positions r_j are measured from the centroid
of the sites (the centre of mass of a homogeneous target): the torque is about that point.
"""
from __future__ import annotations

import numpy as np

from . import interaction


def _centered(r):
    r = np.asarray(r, dtype=np.float64)
    return r - r.mean(axis=0)


def field_tensor(rvec, k):
    """G(R): the field at R of a unit point dipole at the origin is G(R) p (minus the matrix block A_jk)."""
    return -interaction.green_block(rvec, k)


def direct_force_torque(kd, r, p, e_inc, k_tf):
    """Total time-averaged force and torque (about the centroid) on the dipoles, summed site by site
    from the incident field, the full field of every other dipole and each dipole's radiation
    reaction (2/3) i k^3 P_j.  The gradients of the dipole-dipole field are central differences
    with one Richardson step.  O(N^2): tiny targets only.  p, e_inc: (3, N); k_tf: (3,).
    Returns (F, Gamma), real 3-vectors in the Target Frame."""
    k = float(kd)
    rc = _centered(r)
    n = rc.shape[0]
    pt = p.T  # (N, 3)
    et = e_inc.T
    khat = np.asarray(k_tf, float) / np.linalg.norm(k_tf)

    def fld(rvec):  # (..., 3, 3) field tensor at separations rvec (all nonzero)
        return field_tensor(rvec, k)

    def dfld(rvec, c, h):
        e = np.zeros(3)
        e[c] = h
        return (fld(rvec + e) - fld(rvec - e)) / (2.0 * h)

    F = np.zeros(3)
    G = np.zeros(3)
    for j in range(n):
        others = np.arange(n) != j
        R = rc[j][None, :] - rc[others]                     # (N-1, 3)
        E = np.einsum("kab,kb->a", fld(R), pt[others]) + (2.0 / 3.0) * 1j * k ** 3 * pt[j] + et[j]
        gradE = np.zeros((3, 3), dtype=np.complex128)       # gradE[c, a] = d E_a / d r_c
        for c in range(3):
            d1 = dfld(R, c, 1e-3)
            d2 = dfld(R, c, 5e-4)
            gradE[c] = np.einsum("kab,kb->a", (4.0 * d2 - d1) / 3.0, pt[others])
        gradE += np.outer(1j * k * khat, et[j])             # incident field: grad E_a = i k E_a
        f_j = 0.5 * np.real(gradE.conj() @ pt[j])          # 1/2 Re sum_a P_a grad E_a^*
        F += f_j
        G += 0.5 * np.real(np.cross(pt[j], np.conj(E))) + np.cross(rc[j], f_j)
    return F, G


def far_field_force_torque(kd, r, p, e_inc, k_tf, dirs_tf, weights):
    """Force and torque (about the centroid) from the incident part written site by site and the
    array's own part as the far-field integrals above, on the quadrature (dirs_tf: (M, 3) unit
    vectors in the TF, weights: (M,) solid angles).  Returns (F, Gamma) in the TF."""
    k = float(kd)
    rc = _centered(r)
    pt = p.T
    et = e_inc.T
    khat = np.asarray(k_tf, float) / np.linalg.norm(k_tf)
    # incident part
    pe = np.sum(pt * np.conj(et), axis=1)                   # P_j . E_j^*
    F_ext = 0.5 * k * np.sum(np.imag(pe)) * khat
    G_ext = 0.5 * np.sum(np.real(np.cross(pt, np.conj(et))), axis=0) + \
        0.5 * k * np.cross(np.sum(rc * np.imag(pe)[:, None], axis=0), khat)
    F_s = np.zeros(3)
    G_s = np.zeros(3)
    for nv, w in zip(np.asarray(dirs_tf, float), weights):
        ph = np.exp(-1j * k * (rc @ nv))                    # centred positions: a common phase only
        g = pt.T @ ph                                       # (3,)
        f = g - nv * np.dot(nv, g)
        T = (rc * ph[:, None]).T @ pt                       # T[c, a] = sum_j r_jc P_ja e^{...}
        h = T @ np.conj(f)
        F_s -= k ** 4 / (8 * np.pi) * w * np.real(np.vdot(f, f)) * nv
        G_s += k ** 3 / (8 * np.pi) * w * np.imag(np.cross(g, np.conj(f)))
        G_s -= k ** 4 / (8 * np.pi) * w * np.cross(np.real(h), nv)
    return F_ext + F_s, G_ext + G_s


def efficiency_vectors(kd, aeff, F, G):
    """(Q_pr, Q_Gamma) from force and torque: Q = F / (pi a^2 u_rad), k Gamma / (pi a^2 u_rad),
    u_rad = 1 / 8 pi."""
    scale = 8.0 / (aeff * aeff)
    return scale * np.asarray(F), scale * float(kd) * np.asarray(G)


def guide_directions_tf(x, eta, axes):
    """The guide's scattering directions for averaging (observables.scattering_angles) as TF unit
    vectors, with their solid-angle weights."""
    from . import observables, orientation
    dirs, w = [], []
    for th, phis, wt in observables.scattering_angles(x, eta):
        for ph in phis:
            n_lf, _, _ = orientation.scattering_basis_lf(th, ph)
            dirs.append(orientation.lf_to_tf(n_lf, axes))
            w.append(wt)
    return np.array(dirs), np.array(w)


def gauss_directions(n_theta=48, n_phi=96):
    """Product quadrature on the sphere (Gauss-Legendre in cos theta, uniform in phi): exact for
    smooth integrands far beyond the guide's direction sets; used by the pins."""
    xg, wg = np.polynomial.legendre.leggauss(n_theta)
    dirs, w = [], []
    for ct, wc in zip(xg, wg):
        st = np.sqrt(max(0.0, 1.0 - ct * ct))
        for m in range(n_phi):
            ph = 2 * np.pi * (m + 0.5) / n_phi
            dirs.append([st * np.cos(ph), st * np.sin(ph), ct])
            w.append(wc * 2 * np.pi / n_phi)
    return np.array(dirs), np.array(w)

"""Cross sections, scattering amplitudes and Mueller matrix.

Efficiencies (guide, "Introduction": Q = C / (pi a_eff^2), Q_ext = Q_sca + Q_abs;
formulas for C from Draine 1988, which the guide cites), lattice units, |E0| = 1:

    C_ext = 4 pi k sum_j Im(E_inc,j^* . P_j)
    C_abs = 4 pi k sum_j { Im[P_j . (alpha_j^{-1})^* P_j^*] - (2/3) k^3 |P_j|^2 }
    C_pha = 2 pi k sum_j Re(E_inc,j^* . P_j)
    C_sca = C_ext - C_abs

Scattering amplitudes (guide, eq. f_ml_def): with the far field of the dipole
array, f_ml = k^3 sum_j (e_m . P_j^(l)) exp(-i k n_s . r_j), e_1 = theta_hat_s,
e_2 = phi_hat_s.  S_1..S_4 from f_ml with a, b, c, d (guide, the four GETMUELLER
relations), Mueller S_ij (guide, the 16 Bohren & Huffman relations),
dC_sca/dOmega = S_11 / k^2 for unpolarized light, Q_bk = (dC_sca/dOmega at
theta = pi) / (pi a_eff^2).

Angular averages (guide, "Averaging over Scattering Directions"): theta_j
equally spaced in s(theta) = theta + theta/(theta + theta0), theta0 = 2 pi/(1+x),
N_theta from eta, N_phi(j) per ring, solid-angle weights Omega_jk.  The guide
gives N_theta as a real expression without its rounding; this oracle rounds it
to the nearest integer, a reading pinned by the worked example's printed
number of directions.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import orientation as ori_mod


def efficiencies(kd, aeff, e_inc, p, inv_alpha_diag):
    """Q_ext, Q_abs, Q_sca, Q_pha for one RHS. e_inc, p: (3, N); inv_alpha_diag: (N, 3)."""
    k = kd
    c_ext = 4.0 * np.pi * k * np.sum(np.imag(np.conj(e_inc) * p))
    pt = p.T
    # P_j . (alpha_j^{-1})^* P_j^*  (diagonal (N, 3) or full (N, 3, 3) alpha^{-1})
    if inv_alpha_diag.ndim == 2:
        quad = np.sum(pt * np.conj(inv_alpha_diag) * np.conj(pt), axis=1)
    else:
        quad = np.einsum("ja,jab,jb->j", pt, np.conj(inv_alpha_diag), np.conj(pt))
    c_abs = 4.0 * np.pi * k * np.sum(np.imag(quad) - (2.0 / 3.0) * k ** 3 * np.sum(np.abs(pt) ** 2, axis=1))
    c_pha = 2.0 * np.pi * k * np.sum(np.real(np.conj(e_inc) * p))
    geo = np.pi * aeff ** 2
    q_ext, q_abs, q_pha = c_ext / geo, c_abs / geo, c_pha / geo
    return {"Qext": q_ext, "Qabs": q_abs, "Qsca": q_ext - q_abs, "Qpha": q_pha}


def far_field_amplitudes(kd, r, p_pols, theta_s, phi_s, axes):
    """f_ml for one direction (LFRAME angles). p_pols: list of (3, N) solutions, l = 1, 2."""
    n_lf, th_lf, ph_lf = ori_mod.scattering_basis_lf(theta_s, phi_s)
    n_tf = ori_mod.lf_to_tf(n_lf, axes)
    basis_tf = [ori_mod.lf_to_tf(th_lf, axes), ori_mod.lf_to_tf(ph_lf, axes)]
    phase = np.exp(-1j * kd * (r @ n_tf))
    f = np.zeros((2, len(p_pols)), dtype=np.complex128)
    for l, p in enumerate(p_pols):
        for m, e in enumerate(basis_tf):
            f[m, l] = kd ** 3 * np.sum((e @ p) * phase)
    return f


def amplitude_matrix(f, e01_lf, e02_lf, phi_s):
    """S_1..S_4 from f_ml (guide's GETMUELLER relations)."""
    y = np.array([0.0, 1.0, 0.0])
    z = np.array([0.0, 0.0, 1.0])
    a = np.dot(np.conj(e01_lf), y)
    b = np.dot(np.conj(e01_lf), z)
    c = np.dot(np.conj(e02_lf), y)
    d = np.dot(np.conj(e02_lf), z)
    cp, sp = np.cos(phi_s), np.sin(phi_s)
    f11, f12, f21, f22 = f[0, 0], f[0, 1], f[1, 0], f[1, 1]
    s1 = -1j * (f21 * (b * cp - a * sp) + f22 * (d * cp - c * sp))
    s2 = -1j * (f11 * (a * cp + b * sp) + f12 * (c * cp + d * sp))
    s3 = 1j * (f11 * (b * cp - a * sp) + f12 * (d * cp - c * sp))
    s4 = 1j * (f21 * (a * cp + b * sp) + f22 * (c * cp + d * sp))
    return s1, s2, s3, s4


def mueller(s1, s2, s3, s4) -> np.ndarray:
    """4x4 Mueller matrix from the amplitude matrix (Bohren & Huffman relations)."""
    c = np.conj
    m = np.zeros((4, 4))
    m[0, 0] = (abs(s1) ** 2 + abs(s2) ** 2 + abs(s3) ** 2 + abs(s4) ** 2) / 2
    m[0, 1] = (abs(s2) ** 2 - abs(s1) ** 2 + abs(s4) ** 2 - abs(s3) ** 2) / 2
    m[0, 2] = np.real(s2 * c(s3) + s1 * c(s4))
    m[0, 3] = np.imag(s2 * c(s3) - s1 * c(s4))
    m[1, 0] = (abs(s2) ** 2 - abs(s1) ** 2 + abs(s3) ** 2 - abs(s4) ** 2) / 2
    m[1, 1] = (abs(s1) ** 2 + abs(s2) ** 2 - abs(s3) ** 2 - abs(s4) ** 2) / 2
    m[1, 2] = np.real(s2 * c(s3) - s1 * c(s4))
    m[1, 3] = np.imag(s2 * c(s3) + s1 * c(s4))
    m[2, 0] = np.real(s2 * c(s4) + s1 * c(s3))
    m[2, 1] = np.real(s2 * c(s4) - s1 * c(s3))
    m[2, 2] = np.real(s1 * c(s2) + s3 * c(s4))
    m[2, 3] = np.imag(s2 * c(s1) + s4 * c(s3))
    m[3, 0] = np.imag(s4 * c(s2) + s1 * c(s3))
    m[3, 1] = np.imag(s4 * c(s2) - s1 * c(s3))
    m[3, 2] = np.imag(s1 * c(s2) - s3 * c(s4))
    m[3, 3] = np.real(s1 * c(s2) - s3 * c(s4))
    return m


def mueller_for_directions(kd, r, p_pols, dirs, axes, e01_lf, e02_lf):
    """Mueller matrices (ndir, 4, 4) for LFRAME directions dirs = [(theta, phi), ...]."""
    out = np.zeros((len(dirs), 4, 4))
    for i, (th, ph) in enumerate(dirs):
        f = far_field_amplitudes(kd, r, p_pols, th, ph, axes)
        out[i] = mueller(*amplitude_matrix(f, e01_lf, e02_lf, ph))
    return out


def scattering_angles(x: float, eta: float):
    """theta_j, and for each ring the phi values and solid-angle weights Omega_jk."""
    theta0 = 2.0 * np.pi / (1.0 + x)
    n_theta_real = 1.0 + 2.0 * (3.0 + x) / eta * (1.0 + 1.0 / (np.pi + theta0)) / \
        (1.0 + theta0 / (np.pi + theta0) ** 2)
    n_theta = int(np.rint(n_theta_real))
    j = np.arange(1, n_theta + 1)
    s = (j - 1) * np.pi / (n_theta - 1) * (1.0 + 1.0 / (np.pi + theta0))
    theta = ((s - 1.0 - theta0) + np.sqrt((1.0 + theta0 - s) ** 2 + 4.0 * theta0 * s)) / 2.0
    theta[0] = 0.0
    theta[-1] = np.pi
    rings = []
    for jj in range(n_theta):
        if jj == 0 or jj == n_theta - 1:
            nphi = 1
        else:
            nphi = max(3, int(np.rint(4.0 * np.pi * np.sin(theta[jj]) / (theta[jj + 1] - theta[jj - 1]))))
        if jj == 0:
            w = 2.0 * np.pi / nphi * (1.0 - (np.cos(theta[0]) + np.cos(theta[1])) / 2.0)
        elif jj == n_theta - 1:
            w = 2.0 * np.pi / nphi * ((np.cos(theta[-2]) + np.cos(theta[-1])) / 2.0 + 1.0)
        else:
            w = np.pi / nphi * (np.cos(theta[jj - 1]) - np.cos(theta[jj + 1]))
        phis = 2.0 * np.pi * np.arange(nphi) / nphi
        rings.append((theta[jj], phis, w))
    return rings


def angular_averages(kd, r, p, axes, x, eta, e_pol_lf=None):
    """Q_sca by integration of the scattered intensity, and <cos theta>, <cos^2 theta>.

    Scattered intensity for one solution p (one incident polarization):
    dC_sca/dOmega = k^4 |sum_j (P_j - n (n.P_j)) exp(-i k n.r_j)|^2.
    Returns (C_sca_int, g1 = <cos>, g2 = <cos^2>, g_vec (3,) in LF, n_dirs).
    """
    rings = scattering_angles(x, eta)
    c_sca = 0.0
    gc = 0.0
    gc2 = 0.0
    gv = np.zeros(3)
    ndir = 0
    for th, phis, w in rings:
        for ph in phis:
            n_lf, th_lf, ph_lf = ori_mod.scattering_basis_lf(th, ph)
            n_tf = ori_mod.lf_to_tf(n_lf, axes)
            phase = np.exp(-1j * kd * (r @ n_tf))
            fvec = p @ phase  # (3,) sum_j P_j exp(-ik n.r_j)
            fperp = fvec - n_tf * np.dot(n_tf, fvec)
            dcs = kd ** 4 * np.real(np.vdot(fperp, fperp))
            c_sca += dcs * w
            gc += dcs * w * np.cos(th)
            gc2 += dcs * w * np.cos(th) ** 2
            gv += dcs * w * n_lf
            ndir += 1
    return c_sca, gc / c_sca, gc2 / c_sca, gv / c_sca, ndir

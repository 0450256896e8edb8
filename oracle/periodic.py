"""Targets periodic in the Target Frame's y and/or z direction (guide, "Target Generation: Periodic
Targets" and "Interaction Cutoff Parameter for PBC Calculations"; Draine & Flatau 2008).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A Target Unit Cell (TUC) of N dipoles repeats with periods P_y (along y_TF) and/or P_z (along z_TF)
(a period of 0: no repetition along that axis).  Under a plane wave with wave vector k (TF), the
replica displaced by R = m P_y y + n P_z z carries the TUC's polarization times exp(i k.R), so the
equations close on the TUC:

    alpha_j^{-1} P_j + sum_k A^per(r_j - r_k) P_k = E_inc,j,
    A^per(r) = sum_R exp(i k.R) A(r - R) phi(|r - R|)      (the term r - R = 0 omitted),

with A the finite-target block (interaction.green_block).  The lattice sum converges only
conditionally; the guide's parameter gamma tames it with a smooth cutoff phi whose form the guide
leaves to Draine & Flatau (2008).  Reading taken here:

    phi(r) = exp[-(gamma k r)^4],

summed over every replica with (gamma k |R|)^4 <= 40 (beyond that the factor is below 4e-18).
For r = 0 (a site and its own images) only R != 0 contributes.  A^per is not even in r unless
k.R vanishes for every R (normal incidence), so the FFT embedding below fills every offset.
"""
from __future__ import annotations

import numpy as np

from . import interaction

CUTOFF_EXP = 40.0   # (gamma k |R|)^4 above which replicas are dropped


def replica_offsets(periods, kd, gamma, extra=0.0):
    """Replica displacement vectors R (M, 3) covering |R| <= r_max + extra, with their indices."""
    py, pz = periods
    rmax = CUTOFF_EXP ** 0.25 / (gamma * kd) + extra
    my = int(np.ceil(rmax / py)) if py > 0 else 0
    mz = int(np.ceil(rmax / pz)) if pz > 0 else 0
    m, n = np.meshgrid(np.arange(-my, my + 1), np.arange(-mz, mz + 1), indexing="ij")
    R = np.stack([np.zeros(m.size), m.ravel() * float(py), n.ravel() * float(pz)], axis=1)
    keep = np.linalg.norm(R, axis=1) <= rmax
    return R[keep]


def green_per(rvec, kd, k_tf, periods, gamma):
    """A^per at separations rvec (..., 3): (..., 3, 3) complex."""
    rvec = np.asarray(rvec, dtype=np.float64)
    shp = rvec.shape[:-1]
    flat = rvec.reshape(-1, 3)
    ext = float(np.max(np.linalg.norm(flat, axis=1))) if flat.size else 0.0
    R = replica_offsets(periods, kd, gamma, extra=ext)
    ph = np.exp(1j * (R @ np.asarray(k_tf, float)))
    out = np.zeros((flat.shape[0], 3, 3), dtype=np.complex128)
    for i, r in enumerate(flat):
        d = r[None, :] - R
        dist = np.linalg.norm(d, axis=1)
        ok = dist > 0
        w = ph[ok] * np.exp(-(gamma * kd * dist[ok]) ** 4)
        out[i] = np.einsum("m,mab->ab", w, interaction.green_block(d[ok], kd))
    return out.reshape(shp + (3, 3))


def matvec_direct(r, kd, inv_alpha, p, k_tf, periods, gamma):
    """(A p) for the periodic target by the plain O(N^2 x replicas) sum; p (3, N)."""
    n = r.shape[0]
    pt = p.T
    out = np.zeros((3, n), dtype=np.complex128)
    for j in range(n):
        blocks = green_per(r[j][None, :] - r, kd, k_tf, periods, gamma)   # (N, 3, 3), the self term included
        out[:, j] = np.einsum("kab,kb->a", blocks, pt)
    return out + interaction.diagonal_term(inv_alpha, p)


def green_grid(box, pad, kd, k_tf, periods, gamma):
    """A^per on the wrapped padded grid, (3, 3, Pz, Py, Px), every reachable offset filled."""
    nx, ny, nz = box
    px, py, pz = pad
    g = np.zeros((3, 3, pz, py, px), dtype=np.complex128)
    ox = np.arange(-(nx - 1), nx)
    oy = np.arange(-(ny - 1), ny)
    oz = np.arange(-(nz - 1), nz)
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    rvec = np.stack([X, Y, Z], axis=-1).astype(np.float64)
    blk = green_per(rvec, kd, k_tf, periods, gamma)
    gi = np.ix_(oz % pz, oy % py, ox % px)
    for a in range(3):
        for b in range(3):
            g[a, b][gi] = blk[..., a, b]
    return g


def matvec_fft(ijk, box, kd, inv_alpha, p, k_tf, periods, gamma, pad=None, ghat=None):
    """(A p) for the periodic target via the zero-padded FFT convolution with A^per."""
    import scipy.fft as sfft
    pad = interaction.default_pad(box) if pad is None else tuple(pad)
    if ghat is None:
        ghat = sfft.fftn(green_grid(box, pad, kd, k_tf, periods, gamma), axes=(2, 3, 4))
    px, py, pz = pad
    ix, iy, iz = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    phat = []
    for b in range(3):
        grid = np.zeros((pz, py, px), dtype=np.complex128)
        grid[iz, iy, ix] = p[b]
        phat.append(sfft.fftn(grid))
    out = np.empty_like(p, dtype=np.complex128)
    for a in range(3):
        acc = ghat[a, 0] * phat[0] + ghat[a, 1] * phat[1] + ghat[a, 2] * phat[2]
        out[a] = sfft.ifftn(acc)[iz, iy, ix]
    return out + interaction.diagonal_term(inv_alpha, p)


def slab_fresnel_absorption(m, kd, nlayers):
    """Fraction of normally incident power absorbed by a homogeneous slab of index m and thickness
    nlayers d in vacuum (Airy summation of the Fresnel amplitudes; Born & Wolf, section 1.6)."""
    n0, n1 = 1.0, complex(m)
    r01 = (n0 - n1) / (n0 + n1)
    r12 = (n1 - n0) / (n1 + n0)
    t01 = 2 * n0 / (n0 + n1)
    t12 = 2 * n1 / (n1 + n0)
    beta = kd * n1 * nlayers
    e2 = np.exp(2j * beta)
    r = (r01 + r12 * e2) / (1 + r01 * r12 * e2)
    t = t01 * t12 * np.exp(1j * beta) / (1 + r01 * r12 * e2)
    return 1.0 - abs(r) ** 2 - abs(t) ** 2


# ----------------------------------------------------------------------------- scattering into orders
# Guide, "Scattering Directions for Targets that are Periodic in 1 Dimension", "Scattering Directions
# for Doubly-Periodic Targets" and "Scattering by Periodic Targets: Generalized Mueller Matrix" (the
# guide defers the normalisation to Draine & Flatau 2008; the readings below are derived here).
#
# Far from a doubly periodic target (cell area A = P_y P_z), the replicas' dipoles P_j exp(i k.R) add
# up to plane waves, one per allowed order (M, N) on each side of the slab.  Summing the dipole far
# field k^2 (I - n n).P exp(ik|r - r_j - R|)/|r - r_j - R| over the replicas (Weyl's plane-wave form of
# exp(ikR)/R, or the lattice Poisson sum) gives for the order with unit vector n:
#     E_s = (2 pi i k^2 / (A k_x,s)) (I - n n).F e^{i k n.r},   F = sum_j P_j exp(-i k n.r_j),
# k_x,s = k |n_x|.  The finite-target far field of the same F is k^2 (I - n n).F e^{ikr}/r, so the
# order's amplitude is the finite-target amplitude with 1/(kr) replaced by 2 pi/(A k k_x,s); hence
#     S^(2d)_ij(M, N) = S_ij(n) (2 pi / (A k k_x,s))^2,
# S_ij(n) the finite-target Mueller matrix of the same solutions in direction n, and I_sca = S^(2d) I_in
# (the guide's relation, Stokes vectors as intensities of the plane waves).  For a target periodic
# along one axis (period L) the replicas sum to cylindrical waves on the cone of order M:
#     E_s = k^2 (I - n n).F (1/L) i pi H_0^(1)(k_perp rho) ~ k^2 (I - n n).F sqrt(2 pi/(k_perp rho)) / L
# in magnitude (rho: distance from the axis, k_perp = (k^2 - k_axis^2)^(1/2)), so with the guide's
# I_sca = S^(1d) I_in / (k rho)
#     S^(1d)_ij(M, zeta) = S_ij(n) 2 pi / (k k_perp L^2).
# The scattered Stokes vectors exclude the incident wave; the transmission coefficient of order
# (0, 0) includes it: T = |e + E_s|^2 (|n_x| / |n0_x|), R = |E_s|^2 (|n_x| / |n0_x|) for the other
# orders and for reflection (power per unit area of the slab, incident power per unit area |n0_x|).


def order_direction(k_tf, periods, M, N=0, zeta=0.0, sign=1):
    """Unit scattering direction (TF components) of an allowed order of a periodic target, or None
    when the order is evanescent.  Doubly periodic: order (M, N); sign = +1 transmission (k_x of the
    incident wave's sign), -1 reflection.  Singly periodic: order M along the repetition axis and
    azimuth zeta around it (right-handed): axis y -> (k_perp cos zeta, k_y, k_perp sin zeta); axis z
    -> (k_perp cos zeta, k_perp sin zeta, k_z)."""
    k = np.asarray(k_tf, float)
    kd = float(np.linalg.norm(k))
    py, pz = periods
    if py > 0 and pz > 0:
        ky = k[1] + 2.0 * np.pi * M / py
        kz = k[2] + 2.0 * np.pi * N / pz
        kx2 = kd * kd - ky * ky - kz * kz
        if kx2 <= 0.0:
            return None
        sx = 1.0 if k[0] >= 0.0 else -1.0
        return np.array([sign * sx * np.sqrt(kx2), ky, kz]) / kd
    if py > 0:
        ka = k[1] + 2.0 * np.pi * M / py
    else:
        ka = k[2] + 2.0 * np.pi * M / pz
    kp2 = kd * kd - ka * ka
    if kp2 <= 0.0:
        return None
    kp = np.sqrt(kp2)
    if py > 0:
        return np.array([kp * np.cos(zeta), ka, kp * np.sin(zeta)]) / kd
    return np.array([kp * np.cos(zeta), kp * np.sin(zeta), ka]) / kd


def order_sum(r, kd, p, n):
    """F = sum_j P_j exp(-i k n.r_j) for one solution p (3, N): (3,) complex."""
    return p @ np.exp(-1j * kd * (r @ n))


def mueller_in_order(prob, o, ps, n):
    """S^(2d) (doubly periodic) or S^(1d) (singly periodic) of orientation o (RHS 2o and 2o+1, iorth = 2)
    in TF direction n."""
    from . import observables
    rh = prob.rhs[2 * o]
    ax = rh.axes
    n_lf = np.array([np.dot(n, ax[0]), np.dot(n, ax[1]), np.dot(n, ax[2])])
    theta = float(np.arccos(np.clip(n_lf[0], -1.0, 1.0)))
    # along +-x_LF (the (0, 0) orders) the scattering plane is undefined: azimuth 0 there
    phi = float(np.arctan2(n_lf[2], n_lf[1])) if np.hypot(n_lf[1], n_lf[2]) > 1e-9 else 0.0
    kd = prob.kd
    f = observables.far_field_amplitudes(kd, prob.target.r, [ps[2 * o], ps[2 * o + 1]], theta, phi, ax)
    s = observables.mueller(*observables.amplitude_matrix(f, rh.e01_lf, rh.e02_lf, phi))
    py, pz = prob.periods
    if py > 0 and pz > 0:
        return s * (2.0 * np.pi / (py * pz * kd * kd * abs(n[0]))) ** 2
    length = py if py > 0 else pz
    n_axis = n[1] if py > 0 else n[2]
    k_perp = kd * np.sqrt(max(0.0, 1.0 - n_axis * n_axis))
    return s * 2.0 * np.pi / (kd * k_perp * length * length)


def order_fields(prob, i, p, M, N):
    """(E_t, E_r): complex amplitude vectors of order (M, N) of a doubly periodic target for RHS i, the
    transmitted one including the incident wave for (0, 0); far from the slab the field is
    sum over orders of E exp(i k n.x) (incident amplitude e_tf, |E0| = 1).  None if evanescent."""
    rh = prob.rhs[i]
    kd = prob.kd
    area = prob.periods[0] * prob.periods[1]
    out = []
    for sign in (1, -1):
        n = order_direction(rh.k_tf, prob.periods, M, N, sign=sign)
        if n is None:
            return None
        F = order_sum(prob.target.r, kd, p, n)
        E = 2j * np.pi * kd * kd / (area * kd * abs(n[0])) * (F - n * np.dot(n, F))
        if sign == 1 and M == 0 and N == 0:
            E = E + rh.e_tf
        out.append((n, E))
    return tuple(out)


def transmission_reflection(prob, i, p, M, N):
    """(T, R): fractions of the incident power per unit area of a doubly periodic target carried by
    order (M, N) in transmission and in reflection, for RHS i with solution p (3, N); None for an
    evanescent order."""
    rh = prob.rhs[i]
    kd = prob.kd
    py, pz = prob.periods
    area = py * pz
    n0x = abs(rh.k_tf[0]) / kd
    out = []
    for sign in (1, -1):
        n = order_direction(rh.k_tf, prob.periods, M, N, sign=sign)
        if n is None:
            return None
        F = order_sum(prob.target.r, kd, p, n)
        fperp = F - n * np.dot(n, F)
        E = 2j * np.pi * kd * kd / (area * kd * abs(n[0])) * fperp
        if sign == 1 and M == 0 and N == 0:
            E = E + rh.e_tf
        out.append(float(np.real(np.vdot(E, E))) * abs(n[0]) / n0x)
    return tuple(out)


def slab_fresnel_rt(m, kd, nlayers):
    """(R, T) of a homogeneous slab of index m and thickness nlayers d in vacuum at normal incidence
    (the Airy sums of slab_fresnel_absorption)."""
    n0, n1 = 1.0, complex(m)
    r01 = (n0 - n1) / (n0 + n1)
    r12 = (n1 - n0) / (n1 + n0)
    t01 = 2 * n0 / (n0 + n1)
    t12 = 2 * n1 / (n1 + n0)
    beta = kd * n1 * nlayers
    e2 = np.exp(2j * beta)
    r = (r01 + r12 * e2) / (1 + r01 * r12 * e2)
    t = t01 * t12 * np.exp(1j * beta) / (1 + r01 * r12 * e2)
    return abs(r) ** 2, abs(t) ** 2

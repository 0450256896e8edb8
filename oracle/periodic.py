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

"""The DDA matrix A of A P = E (guide, eq. AP=E) and its products.

The guide states the linear system and delegates A to Draine (1988).  For the
point dipoles j != k with r = r_j - r_k, r = |r|, rhat = r / r (lattice units,
k = kd):

    A_jk = exp(i k r) / r * [ k^2 (rhat rhat - I) + (i k r - 1) / r^2 (3 rhat rhat - I) ]

which is minus the field at j radiated by a unit dipole at k, so that
alpha_j^{-1} P_j + sum_{k != j} A_jk P_k = E_inc,j.  The diagonal block is
A_jj = alpha_j^{-1} (diagonal here).

Three ways to apply A, all FP64:
  dense_matrix   the full 3N x 3N matrix (tiny targets, LU);
  matvec_direct  the O(N^2) sum, chunked over rows;
  matvec_fft     the zero-padded FFT convolution of Goodman, Draine & Flatau
                 (1991): the off-diagonal part is a discrete convolution over
                 lattice offsets, so placing P on a padded grid and multiplying
                 FFT(G) by FFT(P) gives it exactly (up to rounding).
Vectors are complex arrays of shape (3, N): component-major, like the layout of
the CUDA library's buffers.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def diagonal_term(inv_alpha: np.ndarray, p: np.ndarray) -> np.ndarray:
    """alpha_j^{-1} P_j for every site: inv_alpha (N, 3) diagonal or (N, 3, 3) full tensors
    (rotated anisotropic materials); p (3, N) -> (3, N)."""
    if inv_alpha.ndim == 2:
        return inv_alpha.T * p
    return np.einsum("jab,bj->aj", inv_alpha, p)


def diag_block(inv_alpha: np.ndarray, j: int) -> np.ndarray:
    """The 3 x 3 diagonal block A_jj = alpha_j^{-1}."""
    return np.diag(inv_alpha[j]) if inv_alpha.ndim == 2 else inv_alpha[j]


def green_block(rvec: np.ndarray, k: float) -> np.ndarray:
    """A_jk for separation vectors rvec (..., 3) (nonzero). Returns (..., 3, 3) complex."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r = np.sqrt(np.sum(rvec * rvec, axis=-1))
    rhat = rvec / r[..., None]
    rr = rhat[..., :, None] * rhat[..., None, :]
    eye = np.eye(3)
    pref = np.exp(1j * k * r) / r
    term2 = (1j * k * r - 1.0) / (r * r)
    return pref[..., None, None] * (k * k * (rr - eye) + term2[..., None, None] * (3.0 * rr - eye))


def dense_matrix(r: np.ndarray, kd: float, inv_alpha_diag: np.ndarray) -> np.ndarray:
    """Full 3N x 3N matrix, unknown ordering (component, site): index = c * N + j.

    inv_alpha_diag: (N, 3) complex diagonal of alpha_j^{-1}.
    """
    n = r.shape[0]
    a = np.zeros((3, n, 3, n), dtype=np.complex128)
    for j in range(n):
        d = r[j][None, :] - r
        d[j] = 1.0  # placeholder, overwritten below
        blk = green_block(d, kd)  # (N,3,3)
        blk[j] = diag_block(inv_alpha_diag, j)
        a[:, j, :, :] = np.transpose(blk, (1, 2, 0))
    return a.reshape(3 * n, 3 * n)


def matvec_direct(r: np.ndarray, kd: float, inv_alpha_diag: np.ndarray, p: np.ndarray,
                  rows=None, chunk: int = 256) -> np.ndarray:
    """(A p) restricted to `rows` (default all sites) by the plain O(N^2) sum. p: (3, N)."""
    n = r.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.zeros((3, rows.size), dtype=np.complex128)
    pt = p.T  # (N,3)
    for s in range(0, rows.size, chunk):
        rj = rows[s:s + chunk]
        d = r[rj][:, None, :] - r[None, :, :]           # (c, N, 3)
        self_mask = rj[:, None] == np.arange(n)[None, :]
        d[self_mask] = 1.0
        blk = green_block(d, kd)                         # (c, N, 3, 3)
        blk[self_mask] = 0.0
        acc = np.einsum("jkab,kb->ja", blk, pt)
        acc += diagonal_term(inv_alpha_diag[rj], p[:, rj]).T
        out[:, s:s + rj.size] = acc.T
    return out


def default_pad(box) -> tuple:
    """Smallest 2,3,5-smooth length >= 2 N per axis (the guide's extended volume)."""
    def smooth(v):
        while True:
            q = v
            for f in (2, 3, 5):
                while q % f == 0:
                    q //= f
            if q == 1:
                return v
            v += 1
    return tuple(smooth(2 * int(b)) for b in box)


def green_grid(box, pad, kd: float) -> np.ndarray:
    """G_ab on the wrapped padded grid: shape (3, 3, Pz, Py, Px), zero at offset 0.

    Offsets n run over -(N-1)..(N-1) per axis; offset n sits at index n mod P.
    Indices not reachable by any pair of sites stay zero.
    """
    nx, ny, nz = box
    px, py, pz = pad
    g = np.zeros((3, 3, pz, py, px), dtype=np.complex128)
    ox = np.arange(-(nx - 1), nx)
    oy = np.arange(-(ny - 1), ny)
    oz = np.arange(-(nz - 1), nz)
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    rvec = np.stack([X, Y, Z], axis=-1).astype(np.float64)
    zero = (X == 0) & (Y == 0) & (Z == 0)
    rvec[zero] = 1.0
    blk = green_block(rvec, kd)
    blk[zero] = 0.0
    gi = np.ix_(oz % pz, oy % py, ox % px)
    for a in range(3):
        for b in range(3):
            g[a, b][gi] = blk[..., a, b]
    return g


def matvec_fft(ijk: np.ndarray, box, kd: float, inv_alpha_diag: np.ndarray, p: np.ndarray,
               pad=None, ghat=None, workers=None) -> np.ndarray:
    """(A p) via the zero-padded FFT convolution. p: (3, N) complex; returns (3, N)."""
    import scipy.fft as sfft
    pad = default_pad(box) if pad is None else tuple(pad)
    if ghat is None:
        ghat = green_fft(box, pad, kd, workers=workers)
    px, py, pz = pad
    ix, iy, iz = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    phat = []
    for b in range(3):
        grid = np.zeros((pz, py, px), dtype=np.complex128)
        grid[iz, iy, ix] = p[b]
        phat.append(sfft.fftn(grid, workers=workers))
    out = np.empty_like(p, dtype=np.complex128)
    for a in range(3):
        acc = ghat[a, 0] * phat[0] + ghat[a, 1] * phat[1] + ghat[a, 2] * phat[2]
        conv = sfft.ifftn(acc, workers=workers)
        out[a] = conv[iz, iy, ix]
    out += diagonal_term(inv_alpha_diag, p)
    return out


def green_fft(box, pad, kd: float, workers=None) -> np.ndarray:
    """FFT of green_grid over the three spatial axes."""
    import scipy.fft as sfft
    g = green_grid(box, pad, kd)
    return sfft.fftn(g, axes=(2, 3, 4), workers=workers)

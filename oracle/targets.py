"""Lattice targets, restated from the guide's "Target Generation" section.

Sites sit at cell centres of a unit cubic lattice.  Along an axis with L
candidate sites (L = the shape's extent in units of d), site i has coordinate
x = i + 1/2 - L/2 measured from the Target-Frame origin, so the origin is the
centroid (ELLIPSOID, CYLINDER1, HEX_PRISM).  RCTGLPRSM places the origin at
the centre of the upper x face, so its x runs from -SHPAR_1 to 0.

Inclusion is decided in exact integer arithmetic on doubled coordinates
u = 2x (always integers), with ties on the surface counted as inside.
Pinned in the tests by brute-force site counts over exact rationals, an
independent floating-point point-in-hexagon test, cubic symmetry of the
sphere and the guide's worked example (N = 131072).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Target:
    ijk: np.ndarray      # (N,3) int64 lattice indices inside the bounding box, x fastest order
    box: tuple           # (Nx, Ny, Nz) bounding box of the occupied sites
    origin: np.ndarray   # (3,) TF coordinates of lattice index (0,0,0)
    a1: np.ndarray       # target axis 1 in TF
    a2: np.ndarray       # target axis 2 in TF

    @property
    def n(self) -> int:
        return int(self.ijk.shape[0])

    @property
    def r(self) -> np.ndarray:
        """(N,3) TF positions in lattice units."""
        return self.ijk.astype(np.float64) + self.origin[None, :]

    @property
    def aeff(self) -> float:
        """a_eff / d = (3N / 4 pi)^(1/3) (guide, "Target Size a_eff")."""
        return (3.0 * self.n / (4.0 * np.pi)) ** (1.0 / 3.0)


def _centered_doubled(length: int) -> np.ndarray:
    # doubled coordinate of the L cell centres: 2(i + 1/2 - L/2) = 2i + 1 - L
    i = np.arange(length, dtype=np.int64)
    return 2 * i + 1 - length


def _as_int(v, what):
    iv = int(round(float(v)))
    if abs(float(v) - iv) > 1e-12 or iv <= 0:
        raise ValueError(f"{what} must be a positive integer number of lattice spacings, got {v}")
    return iv


def _finish(u3, keep, a1, a2) -> Target:
    """Crop the candidate grid (doubled coordinates u3 per axis) to the occupied box."""
    ux, uy, uz = u3
    mask = keep
    if not mask.any():
        raise ValueError("target has no occupied sites")
    idx = np.nonzero(mask)  # arrays over (iz, iy, ix) because mask is indexed [z, y, x]
    iz, iy, ix = idx
    lo = np.array([ix.min(), iy.min(), iz.min()])
    hi = np.array([ix.max(), iy.max(), iz.max()])
    box = tuple(int(v) for v in (hi - lo + 1))
    ijk = np.stack([ix - lo[0], iy - lo[1], iz - lo[2]], axis=1).astype(np.int64)
    # np.nonzero on a C-ordered [z,y,x] array already yields x-fastest lexicographic order
    origin = np.array([ux[lo[0]], uy[lo[1]], uz[lo[2]]], dtype=np.float64) / 2.0
    return Target(ijk=ijk, box=box, origin=origin, a1=np.asarray(a1, float), a2=np.asarray(a2, float))


def ellipsoid(s1, s2, s3) -> Target:
    """ELLIPSOID: (x/S1)^2 + (y/S2)^2 + (z/S3)^2 <= 1/4; a1 = x_TF, a2 = y_TF."""
    s1, s2, s3 = (_as_int(s, "SHPAR") for s in (s1, s2, s3))
    ux, uy, uz = _centered_doubled(s1), _centered_doubled(s2), _centered_doubled(s3)
    U = ux[None, None, :]
    V = uy[None, :, None]
    W = uz[:, None, None]
    # with u = 2x: (u/S)^2 summed <= 1, multiplied through by (S1 S2 S3)^2
    lhs = U * U * (s2 * s3) ** 2 + V * V * (s1 * s3) ** 2 + W * W * (s1 * s2) ** 2
    keep = lhs <= (s1 * s2 * s3) ** 2
    return _finish((ux, uy, uz), keep, [1, 0, 0], [0, 1, 0])


def rctglprsm(s1, s2, s3) -> Target:
    """RCTGLPRSM: S1 x S2 x S3 block, x_TF in [-S1, 0], y, z centred; a1 = x_TF, a2 = y_TF."""
    s1, s2, s3 = (_as_int(s, "SHPAR") for s in (s1, s2, s3))
    ux = 2 * np.arange(s1, dtype=np.int64) + 1 - 2 * s1
    uy, uz = _centered_doubled(s2), _centered_doubled(s3)
    keep = np.ones((s3, s2, s1), dtype=bool)
    return _finish((ux, uy, uz), keep, [1, 0, 0], [0, 1, 0])


_CYL_AXES = {1: (0, [1, 0, 0], [0, 1, 0]), 2: (1, [0, 1, 0], [0, 0, 1]), 3: (2, [0, 0, 1], [1, 0, 0])}


def cylinder1(s1, s2, s3) -> Target:
    """CYLINDER1: length S1, diameter S2, axis along x/y/z_TF for SHPAR3 = 1/2/3."""
    length, diam = _as_int(s1, "SHPAR1"), _as_int(s2, "SHPAR2")
    axis, a1, a2 = _CYL_AXES[int(s3)]
    ext = [diam, diam, diam]
    ext[axis] = length
    u = [_centered_doubled(e) for e in ext]
    grids = np.meshgrid(u[2], u[1], u[0], indexing="ij")  # [z, y, x]
    comp = {0: grids[2], 1: grids[1], 2: grids[0]}
    radial = [comp[a] for a in range(3) if a != axis]
    # radial distance^2 <= (S2/2)^2  <=>  (2x)^2 + (2y)^2 <= S2^2 ; axial extent is the candidate grid
    keep = radial[0] ** 2 + radial[1] ** 2 <= diam * diam
    return _finish(tuple(u), keep, a1, a2)


# SHPAR3 -> (prism axis a1, face normal a2) as TF axis indices
_HEX_AXES = {1: (0, 1), 2: (0, 2), 3: (1, 0), 4: (1, 2), 5: (2, 0), 6: (2, 1)}


def hex_prism(s1, s2, s3) -> Target:
    """HEX_PRISM: length S1 along a1, vertex-to-vertex S2, a2 normal to a rectangular face.

    In the plane normal to a1, with coordinates p along a2 and q along a3 = a1 x a2,
    the hexagon of side S2/2 has apothem h = S2 sqrt(3)/4 and face normals at 0, 60 and
    120 degrees from a2.  Inside  <=>  |p| <= h  and  |p/2 +- (sqrt3/2) q| <= h.
    With doubled coordinates P = 2p, Q = 2q these become
        4 P^2 <= 3 S2^2   and   2 sqrt3 |P Q| <= a := 3 S2^2 - P^2 - 3 Q^2,
    the latter tested exactly as a >= 0 and 12 P^2 Q^2 <= a^2.
    """
    length, vv = _as_int(s1, "SHPAR1"), _as_int(s2, "SHPAR2")
    ax1, ax2 = _HEX_AXES[int(s3)]
    ax3 = 3 - ax1 - ax2
    e = np.eye(3)
    a1, a2 = e[ax1], e[ax2]
    a3 = np.cross(a1, a2)
    ext = [vv, vv, vv]
    ext[ax1] = length
    u = [_centered_doubled(n) for n in ext]
    grids = np.meshgrid(u[2], u[1], u[0], indexing="ij")
    comp = {0: grids[2], 1: grids[1], 2: grids[0]}
    P = comp[ax2] * int(round(a2[ax2]))
    Q = comp[ax3] * int(round(a3[ax3]))
    a = 3 * vv * vv - P * P - 3 * Q * Q
    keep = (4 * P * P <= 3 * vv * vv) & (a >= 0) & (12 * (P * Q) ** 2 <= a * a)
    return _finish(tuple(u), keep, a1, a2)


def make_target(shape: str, shpar) -> Target:
    shape = shape.upper()
    if shape == "ELLIPSOID":
        return ellipsoid(*shpar[:3])
    if shape == "RCTGLPRSM":
        return rctglprsm(*shpar[:3])
    if shape == "CYLINDER1":
        return cylinder1(*shpar[:3])
    if shape == "HEX_PRISM":
        return hex_prism(*shpar[:3])
    raise ValueError(f"unsupported shape {shape}")


def from_sites(ijk, origin, a1=(1, 0, 0), a2=(0, 1, 0)) -> Target:
    """Target from an explicit site list (the guide's FROM_FILE route): ijk (N,3) ints."""
    ijk = np.asarray(ijk, dtype=np.int64)
    lo = ijk.min(axis=0)
    rel = ijk - lo
    box = tuple(int(v) for v in rel.max(axis=0) + 1)
    order = np.lexsort((rel[:, 0], rel[:, 1], rel[:, 2]))
    return Target(ijk=rel[order], box=box, origin=np.asarray(origin, float) + lo,
                  a1=np.asarray(a1, float), a2=np.asarray(a2, float))

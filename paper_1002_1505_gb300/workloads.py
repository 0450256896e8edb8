"""Seeded synthetic workloads shared by the CUDA path, its tests and the oracle.

This module only *describes* inputs: target shape names and shape parameters
(SHPAR, in lattice units), refractive indices, size parameters, orientation
angles and incident polarization vectors.  It contains none of the method's
arithmetic (no rasterization, no polarizabilities, no fields), so both the
CUDA path and the independent FP64 oracle can consume it without sharing any
computation.

Conventions follow the DDSCAT 7.1 guide:
  * shapes and SHPAR meanings: section "Target Generation" (ELLIPSOID,
    RCTGLPRSM, CYLINDER1, HEX_PRISM);
  * orientation angles (beta, Theta, Phi) of the target in the Lab Frame:
    section "Target Orientation";
  * e01 is the user-given incident polarization in the Lab Frame, IORTH=2
    adds e02 = x_LF x e01*: section "Incident Polarization State".

Random draws use numpy's PCG64 with seed 20100207 and one stream per workload,
so every consumer sees the same numbers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED = 20100207

# e01 = y_LF, the guide's sample choice (Lab-Frame components x, y, z).
E01_Y = ((0.0, 0.0), (1.0, 0.0), (0.0, 0.0))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One DDA problem: a target, a material, a wave and a set of RHS."""

    name: str
    shape: str                      # ELLIPSOID | RCTGLPRSM | CYLINDER1 | HEX_PRISM
    shpar: Tuple[float, ...]        # SHPAR_1.. in lattice units
    m: complex                      # refractive index relative to the medium
    x: float                        # size parameter 2 pi a_eff / lambda
    prescription: str               # CM | LATTDR | GKDLDR
    orientations: Tuple[Tuple[float, float, float], ...]  # (beta, Theta, Phi), radians
    iorth: int = 2
    e01: Tuple[Tuple[float, float], ...] = E01_Y
    pad: Optional[Tuple[int, int, int]] = None  # padded FFT grid, None = auto

    @property
    def n_rhs(self) -> int:
        return len(self.orientations) * self.iorth


def uniform_orientations(n: int, stream: int) -> Tuple[Tuple[float, float, float], ...]:
    """n orientations drawn uniformly on SO(3): cos(Theta)~U[-1,1], Phi, beta~U[0,2pi)."""
    rng = np.random.default_rng([SEED, stream])
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    beta = rng.uniform(0.0, 2.0 * math.pi, n)
    return tuple((float(b), float(math.acos(c)), float(p)) for b, c, p in zip(beta, cos_t, phi))


IDENTITY = ((0.0, 0.0, 0.0),)

# Sphere of diameter 12 d, m = 1.33+0.01i, x = 1, lattice dispersion relation.
SPHERE12 = Workload("sphere12_m1.33_x1", "ELLIPSOID", (12, 12, 12), 1.33 + 0.01j, 1.0,
                    "LATTDR", IDENTITY)

# Triaxial ellipsoid filling a 64x48x32 box, m = 1.5+0.1i, x = 5, FFT grid 128x96x64.
ELLIPSOID64 = Workload("ellipsoid64x48x32_m1.5_x5", "ELLIPSOID", (64, 48, 32), 1.5 + 0.1j, 5.0,
                       "GKDLDR", IDENTITY, pad=(128, 96, 64))

# Rectangular prism 48^3, m = 1.7+0.3i, x = 8, 64 random orientations x 2 polarizations.
PRISM48 = Workload("prism48_m1.7_x8_ori64", "RCTGLPRSM", (48, 48, 48), 1.7 + 0.3j, 8.0,
                   "GKDLDR", uniform_orientations(64, 3))

# Hexagonal prism, length 160 d along z_TF, vertex-to-vertex 128 d, a2 || y_TF (SHPAR3=6),
# m = 1.33+0.001i, x = 20, FFT grid 256x256x320, 16 random orientations x 2 polarizations.
HEXPRISM160 = Workload("hexprism160x128_m1.33_x20_ori16", "HEX_PRISM", (160, 128, 6),
                       1.33 + 0.001j, 20.0, "GKDLDR", uniform_orientations(16, 5),
                       pad=(256, 256, 320))

# The guide's worked example: 0.5x1x1 um Au block as 32x64x64 dipoles at lambda = 0.5 um,
# m = 0.9656+1.8628i, GKDLDR, one orientation, 2 polarizations.  a_eff = 0.49237 um, so
# x = 2 pi a_eff / lambda = 6.187304 (the printed K*AEFF).
AU_BLOCK = Workload("au_block32x64x64", "RCTGLPRSM", (32, 64, 64), 0.9656 + 1.8628j, 6.187304,
                    "GKDLDR", IDENTITY)


def mixed_batch(seed_stream: int = 4) -> List[Workload]:
    """Uneven mixed batch: spheres D=16..64 and three cylinders, |m|kd = 0.5, 2 orientations each.

    x is left at 0 here and fixed by the consumer from |m| kd = 0.5 once N is known
    (x = 0.5/|m| * a_eff/d); only the random orientations are drawn here.
    """
    m = 1.7 + 0.3j
    specs = [("ELLIPSOID", (d, d, d)) for d in (16, 24, 32, 40, 48, 64)]
    specs += [("CYLINDER1", (32, 16, 1)), ("CYLINDER1", (64, 40, 2)), ("CYLINDER1", (20, 48, 3))]
    out = []
    for i, (shape, shpar) in enumerate(specs):
        out.append(Workload(f"mixed{i}_{shape.lower()}_{'x'.join(str(s) for s in shpar)}",
                            shape, shpar, m, 0.0, "GKDLDR",
                            uniform_orientations(2, 100 * seed_stream + i)))
    return out


def random_unet_sample(index: int, max_box: int = 48):
    """One random training/eval problem for the learned warm start.

    Returns (shape, shpar, m, x, orientation) drawn from: spheres, ellipsoids and
    hexagonal prisms on boxes up to max_box^3, Re m in [1.1, 2.5], Im m in [0, 0.5],
    x in [1, 10], one uniform orientation.
    """
    rng = np.random.default_rng([SEED, 4, index])
    kind = int(rng.integers(0, 3))
    if kind == 0:
        d = int(rng.integers(8, max_box + 1))
        shape, shpar = "ELLIPSOID", (d, d, d)
    elif kind == 1:
        dims = tuple(int(v) for v in rng.integers(8, max_box + 1, 3))
        shape, shpar = "ELLIPSOID", dims
    else:
        length = int(rng.integers(8, max_box + 1))
        vv = int(rng.integers(8, max_box + 1))
        shape, shpar = "HEX_PRISM", (length, vv, int(rng.integers(1, 7)))
    m = complex(rng.uniform(1.1, 2.5), rng.uniform(0.0, 0.5))
    x = float(rng.uniform(1.0, 10.0))
    cos_t = rng.uniform(-1.0, 1.0)
    ori = (float(rng.uniform(0, 2 * math.pi)), float(math.acos(cos_t)),
           float(rng.uniform(0, 2 * math.pi)))
    return shape, shpar, m, x, ori


def seeded_vector(shape: Sequence[int], stream: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian test vector (used as a generic P for matvec parity)."""
    rng = np.random.default_rng([SEED, 7, stream])
    v = rng.standard_normal(tuple(shape)) + 1j * rng.standard_normal(tuple(shape))
    return v.astype(dtype)

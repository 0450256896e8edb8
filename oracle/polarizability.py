"""Dipole polarizabilities (guide, "Dipole Polarizabilities").

The guide names the prescriptions but delegates their formulas to
Draine & Goodman (1993, ApJ 405, 685; "LATTDR") and Gutkowicz-Krusin & Draine
(2004, astro-ph/0403082; "GKDLDR").  Restated here, lattice units (d = 1),
k = kd, eps = m^2:

  Clausius-Mossotti     alpha_CM = (3 / 4 pi) (eps - 1) / (eps + 2)
  CM + radiative reaction:
                        1/alpha = 1/alpha_CM - (2/3) i k^3
  LATTDR                1/alpha = 1/alpha_CM + (b1 + eps b2 + eps b3 S) k^2 - (2/3) i k^3,
                        S = sum_a (khat_a e_a)^2 (|e_a|^2 for complex e)
  GKDLDR                diagonal tensor, per Cartesian axis a:
                        1/alpha_aa = 1/alpha_CM + (b1 + eps b2 + eps b3 khat_a^2) k^2 - (2/3) i k^3
  b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004.

Every prescription returns the diagonal of 1/alpha (3 complex numbers) for one
material and one incidence (khat, e).  For real m all three give
Im(1/alpha) = -(2/3) k^3 exactly, which is what makes C_abs vanish.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

B1 = -1.8915316
B2 = 0.1648469
B3 = -1.7700004


def alpha_cm(m: complex) -> complex:
    eps = complex(m) ** 2
    return 3.0 / (4.0 * np.pi) * (eps - 1.0) / (eps + 2.0)


def inv_alpha(prescription: str, m: complex, kd: float, khat, e) -> np.ndarray:
    """Diagonal of alpha^{-1} (3 complex) for refractive index m at lattice wavenumber kd."""
    p = prescription.upper()
    eps = complex(m) ** 2
    inv_cm = 1.0 / alpha_cm(m)
    rr = -(2.0 / 3.0) * 1j * kd ** 3
    khat = np.asarray(khat, float)
    khat = khat / np.linalg.norm(khat)
    if p == "CM":
        return np.full(3, inv_cm + rr, dtype=np.complex128)
    if p == "LATTDR":
        e = np.asarray(e, dtype=np.complex128)
        s = float(np.sum(khat ** 2 * np.abs(e) ** 2))
        val = inv_cm + (B1 + eps * B2 + eps * B3 * s) * kd ** 2 + rr
        return np.full(3, val, dtype=np.complex128)
    if p == "GKDLDR":
        return np.array([inv_cm + (B1 + eps * B2 + eps * B3 * khat[a] ** 2) * kd ** 2 + rr
                         for a in range(3)], dtype=np.complex128)
    raise ValueError(f"unknown prescription {prescription}")

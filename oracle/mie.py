"""Mie series for a homogeneous sphere (Bohren & Huffman 1983, chapter 4).

Written from the textbook equations, not from any program listing:
  psi_n(x) = x j_n(x), chi_n(x) = -x y_n(x), xi_n = psi_n - i chi_n;
  logarithmic derivative D_n(mx) = psi_n'(mx) / psi_n(mx) by downward recurrence
      D_{n-1} = n/(mx) - 1 / (D_n + n/(mx)), started well above n_stop;
  a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
  b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]
  Q_ext  = (2/x^2) sum (2n+1) Re(a_n + b_n)
  Q_sca  = (2/x^2) sum (2n+1) (|a_n|^2 + |b_n|^2)
  Q_back = (1/x^2) |sum (2n+1) (-1)^n (a_n - b_n)|^2
  n_stop = x + 4 x^(1/3) + 2.
The DDSCAT guide (section "Applicability of the DDA") validates the DDA against
exact Mie results for pseudospheres; this is that comparison's reference.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def riccati_bessel(x: float, nmax: int):
    """psi_n(x), chi_n(x) for n = 0..nmax by upward recurrence (real x)."""
    psi = np.zeros(nmax + 1)
    chi = np.zeros(nmax + 1)
    psi_m1, psi_0 = np.cos(x), np.sin(x)
    chi_m1, chi_0 = -np.sin(x), np.cos(x)
    psi[0], chi[0] = psi_0, chi_0
    prev_psi, prev_chi = psi_m1, chi_m1
    for n in range(1, nmax + 1):
        psi[n] = (2 * n - 1) / x * psi[n - 1] - prev_psi
        chi[n] = (2 * n - 1) / x * chi[n - 1] - prev_chi
        prev_psi, prev_chi = psi[n - 1], chi[n - 1]
    return psi, chi


def coefficients(m: complex, x: float):
    nstop = int(np.round(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    mx = complex(m) * x
    nmx = int(max(nstop, abs(mx))) + 16
    d = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        d[n - 1] = n / mx - 1.0 / (d[n] + n / mx)
    psi, chi = riccati_bessel(x, nstop)
    xi = psi - 1j * chi
    n = np.arange(1, nstop + 1)
    dn = d[1:nstop + 1]
    ta = dn / m + n / x
    tb = m * dn + n / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return n, a, b


def efficiencies(m: complex, x: float):
    """Returns dict with Qext, Qsca, Qabs, Qback, g for a sphere."""
    n, a, b = coefficients(m, x)
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qback = np.abs(np.sum((2 * n + 1) * (-1.0) ** n * (a - b))) ** 2 / x ** 2
    # asymmetry parameter (Bohren & Huffman eq. 4.62 style sum)
    gsum = np.sum(n[:-1] * (n[:-1] + 2) / (n[:-1] + 1) *
                  np.real(a[:-1] * np.conj(a[1:]) + b[:-1] * np.conj(b[1:])))
    gsum += np.sum((2 * n + 1) / (n * (n + 1)) * np.real(a * np.conj(b)))
    g = 4.0 / (x ** 2 * qsca) * gsum
    return {"Qext": qext, "Qsca": qsca, "Qabs": qext - qsca, "Qback": qback, "g": g}

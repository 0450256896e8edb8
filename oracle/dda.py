"""End-to-end FP64 DDA used by the tests: target -> incidence -> alpha -> solve -> Q.

Steps in the guide's order (section "Choice of Iterative Algorithm" for the
system A P = E; the other sections as cited in the sibling modules).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import interaction, observables, orientation, polarizability, solvers, targets


@dataclasses.dataclass
class Rhs:
    ori: tuple            # (beta, Theta, Phi)
    pol: int              # 0 or 1 (e01 / e02)
    k_tf: np.ndarray      # (3,) k vector in TF (lattice units)
    e_tf: np.ndarray      # (3,) complex polarization in TF
    e01_lf: np.ndarray
    e02_lf: Optional[np.ndarray]
    axes: tuple           # x_LF, y_LF, z_LF in TF
    inv_alpha: np.ndarray  # (N, 3) complex diagonal of alpha^{-1}, or (N, 3, 3) full tensors
    e_inc: np.ndarray     # (3, N) complex incident field


@dataclasses.dataclass
class Problem:
    target: targets.Target
    kd: float
    x: float
    rhs: List[Rhs]
    pad: tuple
    periods: Optional[tuple] = None   # (P_y, P_z) of a periodic target (0: not periodic along that axis)
    gamma: float = 0.0                # interaction cutoff of the periodic sums


def build_problem(shape, shpar, m, x, prescription, orientations, e01_lf=((0, 0), (1, 0), (0, 0)),
                  iorth=2, pad=None, target=None, kd=None, comp=None, df_angles=None, periods=None,
                  gamma=0.01) -> Problem:
    """comp (optional): per-site composition indices (0-based) in the target's site order, shape
    (N,) for isotropic materials or (N, 3) for one composition per Cartesian axis (the guide's
    ICOMP triple of an anisotropic material whose principal axes are the TF axes); m is then a
    sequence of refractive indices, one per composition.
    df_angles (optional, with comp (N, 3)): per-site (theta_DF, phi_DF, beta_DF) of the Dielectric
    Frame (the guide's ANIFRMFIL target): comp[j, a] is the composition along the principal axis
    e_a, and alpha_j^{-1} = sum_a d_a e_a e_a^T (a full symmetric 3 x 3), d_a the prescription's
    value for that composition with the incidence (khat, e) expressed along e_1, e_2, e_3."""
    tgt = targets.make_target(shape, shpar) if target is None else target
    if kd is None:
        kd = x / tgt.aeff            # k d = x / (a_eff / d)
    else:
        x = kd * tgt.aeff
    e01 = np.array([complex(*c) if isinstance(c, (tuple, list)) else complex(c) for c in e01_lf])
    r = tgt.r
    rhs = []
    for ori in orientations:
        k_tf, pols_tf, pols_lf, axes = orientation.incidence(kd, ori, tgt.a1, tgt.a2, e01, iorth)
        for l, e_tf in enumerate(pols_tf):
            if df_angles is not None:
                cj = np.asarray(comp, dtype=np.int64)
                inv_alpha = np.zeros((tgt.n, 3, 3), dtype=np.complex128)
                for j in range(tgt.n):
                    axes_df = orientation.dielectric_axes(*df_angles[j])
                    kdf = np.array([np.dot(k_tf / kd, ea) for ea in axes_df])
                    edf = np.array([np.dot(e_tf, ea) for ea in axes_df])
                    for a, ea in enumerate(axes_df):
                        d_a = polarizability.inv_alpha(prescription, m[cj[j, a]], kd, kdf, edf)[a]
                        inv_alpha[j] += d_a * np.outer(ea, ea)
            elif comp is None:
                ia = polarizability.inv_alpha(prescription, m, kd, k_tf / kd, e_tf)
                inv_alpha = np.tile(ia, (tgt.n, 1))
            else:
                # one diagonal per composition, then axis a of site j takes composition comp[j, a]
                table = np.array([polarizability.inv_alpha(prescription, mc, kd, k_tf / kd, e_tf) for mc in m])
                cj = np.asarray(comp, dtype=np.int64)
                if cj.ndim == 1:
                    cj = np.repeat(cj[:, None], 3, axis=1)
                inv_alpha = table[cj, np.arange(3)[None, :]]
            e_inc = e_tf[:, None] * np.exp(1j * (r @ k_tf))[None, :]
            rhs.append(Rhs(ori=tuple(ori), pol=l, k_tf=k_tf, e_tf=e_tf, e01_lf=pols_lf[0],
                           e02_lf=pols_lf[1] if iorth == 2 else None, axes=axes,
                           inv_alpha=inv_alpha, e_inc=e_inc))
    pad = interaction.default_pad(tgt.box) if pad is None else tuple(pad)
    per = None if periods is None or (periods[0] <= 0 and periods[1] <= 0) else tuple(float(v) for v in periods)
    return Problem(target=tgt, kd=kd, x=x, rhs=rhs, pad=pad, periods=per, gamma=float(gamma))


def apply_a(prob: Problem, i: int, p: np.ndarray, method: str = "fft", ghat=None, workers=None):
    t = prob.target
    if prob.periods is not None:
        from . import periodic
        rh = prob.rhs[i]
        if method == "direct":
            return periodic.matvec_direct(t.r, prob.kd, rh.inv_alpha, p, rh.k_tf, prob.periods, prob.gamma)
        return periodic.matvec_fft(t.ijk, t.box, prob.kd, rh.inv_alpha, p, rh.k_tf, prob.periods, prob.gamma,
                                   pad=prob.pad, ghat=ghat)
    if method == "direct":
        return interaction.matvec_direct(t.r, prob.kd, prob.rhs[i].inv_alpha, p)
    return interaction.matvec_fft(t.ijk, t.box, prob.kd, prob.rhs[i].inv_alpha, p, pad=prob.pad,
                                  ghat=ghat, workers=workers)


def solve(prob: Problem, method: str = "bicgstab", matvec: str = "fft", tol: float = 1e-10,
          workers=None, maxit: int = 3000):
    """Solve every RHS. method: lu | bicgstab | bicgstab2 | ccg | cocg | qmr_cs.
    Returns list of (3, N) P and iteration counts."""
    t = prob.target
    out, iters = [], []
    ghat = None
    if matvec == "fft" and method != "lu" and prob.periods is None:
        ghat = interaction.green_fft(t.box, prob.pad, prob.kd, workers=workers)
    for i, rh in enumerate(prob.rhs):
        if method == "lu":
            if prob.periods is not None:
                from . import periodic
                blocks = periodic.green_per(t.r[:, None, :] - t.r[None, :, :], prob.kd, rh.k_tf, prob.periods,
                                            prob.gamma)                                  # (N, N, 3, 3)
                for j in range(t.n):
                    blocks[j, j] += interaction.diag_block(rh.inv_alpha, j)
                a = np.transpose(blocks, (2, 0, 3, 1)).reshape(3 * t.n, 3 * t.n)
            else:
                a = interaction.dense_matrix(t.r, prob.kd, rh.inv_alpha)
            p = solvers.lu_solve(a, rh.e_inc.reshape(-1)).reshape(3, t.n)
            out.append(p)
            iters.append(0)
            continue
        shape = rh.e_inc.shape

        def op(v, i=i):
            return apply_a(prob, i, v.reshape(shape), matvec, ghat=ghat, workers=workers).reshape(-1)
        fn = {"bicgstab": solvers.bicgstab, "ccg": solvers.ccg, "cocg": solvers.cocg,
              "qmr_cs": lambda *a, **k: solvers.qmr_cs(*a, **k)[:3],
              "bicgstab2": lambda *a, **k: solvers.bicgstab_l(*a, ell=2, **k)}[method]
        p, it, _ = fn(op, rh.e_inc.reshape(-1), tol=tol, maxit=maxit)
        out.append(p.reshape(shape))
        iters.append(it)
    return out, iters


def cross_sections(prob: Problem, ps):
    t = prob.target
    return [observables.efficiencies(prob.kd, t.aeff, rh.e_inc, p, rh.inv_alpha)
            for rh, p in zip(prob.rhs, ps)]


def mueller(prob: Problem, ps, dirs, ori_index: int = 0):
    """Mueller matrices for LFRAME directions; needs both polarizations of one orientation."""
    i0 = 2 * ori_index
    rh = prob.rhs[i0]
    return observables.mueller_for_directions(prob.kd, prob.target.r, [ps[i0], ps[i0 + 1]], dirs,
                                              rh.axes, rh.e01_lf, rh.e02_lf)

"""Radiative force and torque efficiency vectors on the GPU (dda_force_torque) against the FP64
oracle (oracle/forces.py: the same far-field integrals on the same guide directions, itself pinned
to a site-by-site evaluation with the full dipole field and its gradient) and against the guide's
worked example (Q_sca g(1) printed for the Au block).

Bars: each vector within 2e-5 of the oracle's, relative to the largest efficiency of the RHS
(FP32 far-field sums); the Au block's Q_pr,1 = Q_ext - Q_sca g(1) within 2e-3 of the printed value.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from conftest import load_golden  # noqa: E402
from oracle import dda as odda  # noqa: E402
from oracle import forces as ofor  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


CASES = [
    ("ell_odd_linear", W.Workload("ell_odd", "ELLIPSOID", (7, 5, 9), 1.5 + 0.1j, 2.0, "GKDLDR",
                                  W.uniform_orientations(2, 11))),
    ("hex_circular", W.Workload("hex_c", "HEX_PRISM", (6, 10, 3), 1.7 + 0.4j, 2.5, "LATTDR",
                                W.uniform_orientations(2, 13), e01=((0, 0), (1, 0), (0, 1)))),
    ("block_offcentre_origin", W.Workload("blk", "RCTGLPRSM", (4, 7, 5), 2.0 + 1.0j, 1.8, "CM",
                                          W.uniform_orientations(1, 14))),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_force_and_torque_match_oracle(D, name, w):
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.dda_solve(p, precision="C128", tol=1e-9, maxit=3000)
    qpr, qg, ndir = ctx.dda_force_torque(p, eta=0.5)
    q, _ = ctx.dda_cross_sections(p)
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations, e01_lf=w.e01, iorth=w.iorth)
    pn = p.cpu().numpy()
    for b in range(ctx.nrhs):
        rh = prob.rhs[b]
        dirs, wt = ofor.guide_directions_tf(prob.kd * prob.target.aeff, 0.5, rh.axes)
        assert len(wt) == ndir
        F, G = ofor.far_field_force_torque(prob.kd, prob.target.r, pn[b], rh.e_inc, rh.k_tf, dirs, wt)
        rp, rg = ofor.efficiency_vectors(prob.kd, prob.target.aeff, F, G)
        scale = max(abs(q[b, 0]), 1e-30)
        np.testing.assert_allclose(qpr[b], rp, rtol=0, atol=2e-5 * scale)
        np.testing.assert_allclose(qg[b], rg, rtol=0, atol=2e-5 * scale)
        # the force along khat is Q_ext - Q_sca <cos theta> with the same quadrature
        kh = rh.k_tf / np.linalg.norm(rh.k_tf)
        ang, _ = ctx.dda_angular_averages(p, eta=0.5)
        assert np.dot(qpr[b], kh) == pytest.approx(q[b, 0] - ang[b, 0] * ang[b, 1], rel=1e-6)


def test_au_block_force_against_the_printed_moment(D):
    g, _ = load_golden("au_block_worked_example.txt")
    ctx = D.Context(0)
    D.setup_workload(ctx, W.AU_BLOCK)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000)
    qpr, qg, _ = ctx.dda_force_torque(p, eta=0.1)
    for b in range(2):
        # orientation (0, 0, 0): x_LF = x_TF, the incident direction
        assert qpr[b, 0] == pytest.approx(g["Qext"] - g["Qsca_g1"], rel=2e-3)
        assert abs(qpr[b, 1]) < 1e-3 and abs(qpr[b, 2]) < 1e-3
        # mirror symmetry of the block about y and z with linear polarization along y or z: no torque
        assert np.abs(qg[b]).max() < 1e-4 * g["Qext"]

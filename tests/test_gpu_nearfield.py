"""Fields in or near the target (the guide's DDfield postprocessing) on the GPU: against the FP64
oracle (oracle/nearfield.py) for the same solution at points outside, on the surface of and inside
the target (including points within one lattice spacing of dipoles, where the suppression factor
acts), and against the guide's printed DDfield track for the Au block.

Bars: E and B within 1e-10 of the oracle's, relative to the largest field value (both FP64);
the Au block's E_y within 2e-3 of the printed values (single-precision reference run at TOL 1e-5).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from conftest import load_golden  # noqa: E402
from oracle import dda as odda  # noqa: E402
from oracle import nearfield as onf  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


def test_near_field_matches_oracle(D):
    w = W.Workload("ell_nf", "ELLIPSOID", (9, 7, 6), 1.7 + 0.1j, 2.5, "GKDLDR", W.uniform_orientations(2, 111),
                   e01=((0, 0), (1, 0), (0, 1)))
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.dda_solve(p, precision="C128", tol=1e-8, maxit=2000)
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations, e01_lf=w.e01)
    rng = np.random.default_rng(113)
    sites = prob.target.r
    pts = np.concatenate([
        rng.uniform(-12, 12, size=(20, 3)),                       # around the target
        sites[rng.choice(len(sites), 6, replace=False)],          # on dipoles (their own term skipped)
        sites[rng.choice(len(sites), 6, replace=False)] + rng.uniform(-0.45, 0.45, size=(6, 3)),  # within d
        np.array([[0.0, 0.0, 40.0], [-25.0, 3.0, 1.0]]),          # far
    ])
    E, B = ctx.dda_near_field(p, pts)
    pn = p.cpu().numpy()
    for b in range(ctx.nrhs):
        rh = prob.rhs[b]
        Er, Br = onf.fields_at(pts, prob.kd, sites, pn[b], rh.k_tf, rh.e_tf)
        np.testing.assert_allclose(E[b], Er, rtol=0, atol=1e-10 * np.abs(Er).max())
        np.testing.assert_allclose(B[b], Br, rtol=0, atol=1e-10 * np.abs(Br).max())


def test_near_field_au_block_printed_track(D):
    _, rows = load_golden("au_block_ddfield_track.txt")
    ctx = D.Context(0)
    D.setup_workload(ctx, W.AU_BLOCK)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.dda_solve(p, precision="MIXED", tol=1e-6, maxit=3000)
    pts = np.array([row[:3] for row in rows])
    E, _ = ctx.dda_near_field(p, pts, want_b=False)
    for row, e in zip(rows, E[0]):  # polarization 1 = y_LF
        ref = complex(row[3], row[4])
        assert abs(e[1] - ref) <= 2e-3 * max(abs(ref), 0.1), (row, e[1])
        assert abs(e[0]) < 1e-6 and abs(e[2]) < 1e-6

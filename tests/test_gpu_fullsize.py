"""Full-size parity on the two batched workloads, in the launch configuration the benchmark times
(every right-hand side of the workload in one batch).

* prism 48^3, 64 orientations x 2 polarizations = 128 RHS on the 96^3 grid: every RHS's whole
  product against the oracle's FP64 zero-padded FFT product (itself pinned to the direct O(N^2)
  sum to 1e-13 in the oracle's tests), and Q_ext / Q_abs / Q_sca of four RHS from one batched
  mixed-precision solve against the oracle's BiCGstab solved to 1e-10.
* hexagonal prism 160 x 128 (1,694,720 dipoles), 16 orientations x 2 = 32 RHS on 256 x 256 x 320:
  every RHS at sampled rows (direct O(N^2) rows of the oracle; the rows reach both ends of every
  axis of the box), three RHS as whole vectors against the oracle's FFT product, and Q of the
  first orientation's two RHS from the benchmark's 32-RHS solve against values the oracle wrote
  (tests/golden/hexprism160_q.txt, made by tests/golden/make_hexprism160_q.py).

Bars: complex64 product 1e-5 relative L2 (per RHS), complex128 and double-float 1e-12; Q 1e-4
relative (Q_pha 1e-4 of |Q_ext|, absolute).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from conftest import ROOT, load_golden  # noqa: E402
from oracle import dda as odda  # noqa: E402
from oracle import interaction as oint  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


def _problem(w, orientations=None):
    ori = w.orientations if orientations is None else orientations
    return odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, ori, e01_lf=w.e01, iorth=w.iorth,
                              pad=w.pad)


def _ctx(D, w):
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    return ctx


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_prism48_every_rhs_whole_product(D):
    w = W.PRISM48
    ctx = _ctx(D, w)
    prob = _problem(w)
    assert ctx.nrhs == 128 and ctx.n == prob.target.n
    ghat = oint.green_fft(prob.target.box, prob.pad, prob.kd, workers=-1)
    for dt, tol, dfl in ((torch.complex64, 1e-5, False), (torch.complex128, 1e-12, False),
                         (torch.complex128, 1e-12, True)):
        p = torch.from_numpy(W.seeded_vector((ctx.nrhs, 3, ctx.n), 31)).to(dt).cuda()
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap, double_float=dfl)
        got = ap.cpu().numpy().astype(np.complex128)
        pin = p.cpu().numpy().astype(np.complex128)
        errs = [_rel(got[b], odda.apply_a(prob, b, pin[b], "fft", ghat=ghat, workers=-1)) for b in range(ctx.nrhs)]
        assert max(errs) <= tol, (dt, dfl, int(np.argmax(errs)), max(errs))
        del p, ap


def test_prism48_batched_solve_cross_sections(D):
    """Q of RHS 0, 1 (orientation 0) and 126, 127 (orientation 63) from the batched 128-RHS
    mixed-precision solve against the oracle's BiCGstab to 1e-10 on those two orientations."""
    w = W.PRISM48
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000)
    assert all(r["converged"] == 1 and r["true_rel_resid"] <= 1e-5 for r in reps)
    q, _ = ctx.dda_cross_sections(p)
    prob = _problem(w, [w.orientations[0], w.orientations[63]])
    ps, _ = odda.solve(prob, "bicgstab", tol=1e-10, workers=-1)
    qref = odda.cross_sections(prob, ps)
    for k, b in enumerate((0, 1, 126, 127)):
        for i, key in enumerate(("Qext", "Qabs", "Qsca")):
            assert q[b, i] == pytest.approx(qref[k][key], rel=1e-4), (b, key, q[b, i], qref[k][key])
        assert abs(q[b, 3] - qref[k]["Qpha"]) <= 1e-4 * abs(qref[k]["Qext"]), b


def _spanning_rows(sites, rng, extra=4):
    """Site indices that reach the first and last layer of the box along every axis, plus random ones."""
    rows = {0, len(sites) - 1}
    for a in range(3):
        for v in (sites[:, a].min(), sites[:, a].max()):
            cand = np.flatnonzero(sites[:, a] == v)
            rows.add(int(cand[len(cand) // 2]))
    rows.update(int(v) for v in rng.choice(len(sites), extra, replace=False))
    return np.array(sorted(rows))


def test_hexprism_every_rhs_sampled_rows_and_whole_vectors(D):
    w = W.HEXPRISM160
    ctx = _ctx(D, w)
    prob = _problem(w)
    assert ctx.nrhs == 32 and ctx.n == prob.target.n
    sites, _ = ctx.dda_get_sites()
    np.testing.assert_array_equal(sites, prob.target.ijk)
    rows = _spanning_rows(sites, np.random.default_rng(17))
    ghat = oint.green_fft(prob.target.box, prob.pad, prob.kd, workers=-1)
    for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
        p = torch.from_numpy(W.seeded_vector((ctx.nrhs, 3, ctx.n), 41)).to(dt).cuda()
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        for b in range(ctx.nrhs):
            pb = p[b].cpu().numpy().astype(np.complex128)
            got = ap[b].cpu().numpy().astype(np.complex128)
            ref = oint.matvec_direct(prob.target.r, prob.kd, prob.rhs[b].inv_alpha, pb, rows=rows, chunk=2)
            assert _rel(got[:, rows], ref) <= tol, (dt, b)
            if b in (0, 16, 31):
                whole = odda.apply_a(prob, b, pb, "fft", ghat=ghat, workers=-1)
                assert _rel(got, whole) <= tol, (dt, b, _rel(got, whole))
        del p, ap
        torch.cuda.empty_cache()


def test_hexprism_batched_solve_cross_sections_against_oracle_values(D):
    g, _ = load_golden("hexprism160_q.txt")
    w = W.HEXPRISM160
    ctx = _ctx(D, w)
    assert ctx.n == int(g["N"])
    assert ctx.kd == pytest.approx(g["kd"], rel=1e-14)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000)
    assert all(r["converged"] == 1 and r["true_rel_resid"] <= 1e-5 for r in reps)
    q, _ = ctx.dda_cross_sections(p)
    for b in range(2):
        for i, key in enumerate(("Qext", "Qabs", "Qsca")):
            assert q[b, i] == pytest.approx(g[f"{key}_{b}"], rel=1e-4), (b, key, q[b, i], g[f"{key}_{b}"])
        assert abs(q[b, 3] - g[f"Qpha_{b}"]) <= 1e-4 * abs(g[f"Qext_{b}"]), b

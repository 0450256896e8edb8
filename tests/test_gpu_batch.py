"""Mixed batch of targets of uneven grid sizes solved concurrently (dda_solve_batch)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import dda as odda  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


def _setup(D, w):
    """Context for a mixed-batch member: x chosen so that |m| k d = 0.5."""
    ctx = D.Context(0)
    n, _ = ctx.dda_setup_shape(w.shape, w.shpar)
    kd = 0.5 / abs(w.m)
    ctx.dda_set_incident(kd, w.orientations, [[c[0], c[1]] for c in w.e01], w.iorth)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability(w.prescription, w.m)
    return ctx, kd


def test_mixed_batch_matches_single_solves_and_oracle(D):
    ws = W.mixed_batch()
    ctxs, kds = zip(*[_setup(D, w) for w in ws])
    ps = [torch.zeros((c.nrhs, 3, c.n), dtype=torch.complex128, device="cuda") for c in ctxs]
    reps, sts, overall = D.dda_solve_batch(list(ctxs), ps, precision="MIXED", tol=1e-5, maxit=2000)
    assert overall == D.DDA_OK and all(s == D.DDA_OK for s in sts), sts
    for r in reps:
        assert all(x["converged"] == 1 and x["true_rel_resid"] <= 1e-5 for x in r)
    qb = [c.dda_cross_sections(p)[0] for c, p in zip(ctxs, ps)]
    # the same targets solved one at a time
    for c, q in zip(ctxs, qb):
        p1 = torch.zeros((c.nrhs, 3, c.n), dtype=torch.complex128, device="cuda")
        c.dda_solve(p1, precision="MIXED", tol=1e-5, maxit=2000)
        q1, _ = c.dda_cross_sections(p1)
        np.testing.assert_allclose(q[:, :3], q1[:, :3], rtol=1e-4)
        np.testing.assert_allclose(q[:, 3], q1[:, 3], rtol=0, atol=1e-4 * np.abs(q1[:, 0]).max())
    # the smallest members against the FP64 oracle
    for w, kd, q in zip(ws, kds, qb):
        if w.shpar not in ((16, 16, 16), (24, 24, 24), (32, 16, 1)):
            continue
        prob = odda.build_problem(w.shape, w.shpar, w.m, None, w.prescription, w.orientations, e01_lf=w.e01,
                                  iorth=w.iorth, kd=kd)
        psr, _ = odda.solve(prob, "bicgstab", tol=1e-10, workers=-1)
        qref = odda.cross_sections(prob, psr)
        for b in range(len(qref)):
            for i, key in enumerate(("Qext", "Qabs", "Qsca")):
                assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (w.name, b, key)
            # Q_pha can be near zero: bound its error on the scale of Q_ext
            assert abs(q[b, 3] - qref[b]["Qpha"]) <= 1e-4 * abs(qref[b]["Qext"]), (w.name, b)


def test_batch_rejects_duplicate_contexts(D):
    w = W.mixed_batch()[0]
    ctx, _ = _setup(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    _, _, overall = D.dda_solve_batch([ctx, ctx], [p, p])
    assert overall == D.DDA_EINVAL

"""Targets of anisotropic materials whose dielectric axes are rotated per site (the guide's ANIFRMFIL
target, section "Composite Targets with Anisotropic Constituents"): the full symmetric alpha^{-1}
per site in the product's diagonal term and in the absorption sum, against the FP64 oracle.

Bars: product 1e-12 (complex128) / 1e-5 (complex64) relative L2 against the oracle's direct sum;
Q_ext / Q_abs / Q_sca 1e-4 relative against the oracle's LU solution; zero angles reproduce the
TF-aligned anisotropic target's product to rounding.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import dda as odda  # noqa: E402
from oracle import targets as o_targets  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


def _setup(D, t, comp, ang, m, presc, ori, kd):
    ctx = D.Context(0)
    ctx.dda_setup_target_anifrm(t.ijk, comp + 1, ang, origin=t.origin)
    ctx.dda_set_incident(kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability(presc, m)
    return ctx


@pytest.mark.parametrize("box,presc", [((12, 8, 8), "GKDLDR"), ((9, 7, 6), "LATTDR"), ((8, 8, 8), "CM")],
                         ids=["compile_time_grid_gkdldr", "generic_grid_lattdr", "cube_cm"])
def test_rotated_dielectric_frames_match_oracle(D, box, presc):
    t = o_targets.make_target("ELLIPSOID", box)
    rng = np.random.default_rng(91)
    # a uniaxial inclusion (c-axis along e_1) in an isotropic host, c-axis orientation varying by site
    incl = (t.ijk[:, 0] >= box[0] // 2)
    comp = np.where(incl[:, None], np.array([[1, 2, 2]]), np.array([[0, 0, 0]]))
    ang = np.where(incl[:, None], rng.uniform(0, math.pi, size=(t.n, 3)), 0.0)
    m = [1.33 + 0.01j, 1.9 + 0.3j, 1.5 + 0.05j]
    ori = W.uniform_orientations(1, 93)
    prob = odda.build_problem(None, None, m, 2.5, presc, ori, target=t, comp=comp, df_angles=ang)
    ctx = _setup(D, t, comp, ang, m, presc, ori, prob.kd)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = torch.from_numpy(W.seeded_vector((ctx.nrhs, 3, ctx.n), 95)).to(dt).cuda()
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= tol, (dt, b)
    ps, _ = odda.solve(prob, "lu")
    qref = odda.cross_sections(prob, ps)
    for solver, prec in (("BICGSTAB", "MIXED"), ("COCG", "C128")):
        p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
        reps, _ = ctx.dda_solve(p, solver=solver, precision=prec, tol=1e-7, maxit=3000)
        assert all(r["converged"] == 1 for r in reps)
        q, _ = ctx.dda_cross_sections(p)
        for b in range(ctx.nrhs):
            for i, key in enumerate(("Qext", "Qabs", "Qsca")):
                assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (solver, key, b)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_solve(torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda"), precond="JACOBI")
    assert ei.value.status == D.DDA_EUNSUPPORTED


def test_zero_angles_reproduce_the_aligned_target(D):
    t = o_targets.make_target("ELLIPSOID", (12, 8, 8))
    comp = np.stack([t.ijk[:, 2] % 2, (t.ijk[:, 0] // 3) % 3, np.full(t.n, 1)], axis=1)
    m = [1.5 + 0.1j, 1.33 + 0.01j, 2.2 + 0.6j]
    ori = W.uniform_orientations(2, 97)
    kd = 0.31
    a = D.Context(0)
    a.dda_setup_target(t.ijk, icomp=comp + 1, origin=t.origin)
    a.dda_set_incident(kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    a.dda_build_green_fft()
    a.dda_set_polarizability("GKDLDR", m)
    r = _setup(D, t, comp, np.zeros((t.n, 3)), m, "GKDLDR", ori, kd)
    p = torch.from_numpy(W.seeded_vector((a.nrhs, 3, a.n), 99)).cuda()
    y1, y2 = torch.empty_like(p), torch.empty_like(p)
    a.dda_matvec(p, y1)
    r.dda_matvec(p, y2)
    torch.cuda.synchronize()
    assert (torch.linalg.vector_norm(y1 - y2) / torch.linalg.vector_norm(y1)).item() <= 1e-14

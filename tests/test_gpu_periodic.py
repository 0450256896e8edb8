"""Periodic targets (the guide's periodic-target options with the interaction cutoff gamma) on the
GPU: the periodic Green tensor built by dda_build_green_fft against the FP64 oracle's
(oracle/periodic.py, pinned to the replica-by-replica sum and to the Fresnel absorption of a slab).

Bars: product 1e-12 (complex128) / 1e-5 (complex64) relative L2 against the oracle's periodic FFT
product; Q_ext / Q_abs 1e-4 relative against the oracle's LU solution; the slab's absorbed fraction
within 1 % of the continuum film's.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import dda as odda  # noqa: E402
from oracle import periodic as oper  # noqa: E402
from oracle import targets as o_targets  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


@pytest.mark.parametrize("periods,box", [((7.0, 9.0), (4, 5, 6)), ((8.0, 0.0), (5, 6, 4)), ((0.0, 6.0), (6, 4, 5)),
                                         ((9.0, 10.0), (8, 8, 8))],
                         ids=["2d", "1d_y", "1d_z", "2d_compile_time_grid"])
def test_periodic_product_and_solve_match_oracle(D, periods, box):
    t = o_targets.make_target("ELLIPSOID", box)
    ori = [(0.4, 0.9, 1.3)]  # oblique: the replicas carry Bloch phases
    gamma = 0.1
    prob = odda.build_problem(None, None, 1.6 + 0.15j, 2.0, "GKDLDR", ori, target=t, periods=periods, gamma=gamma)
    ctx = D.Context(0)
    ctx.dda_setup_target(t.ijk, origin=t.origin)
    ctx.dda_set_periodicity(periods[0], periods[1], gamma)
    ctx.dda_set_incident(prob.kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("GKDLDR", 1.6 + 0.15j)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = torch.from_numpy(W.seeded_vector((ctx.nrhs, 3, ctx.n), 121)).to(dt).cuda()
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "fft")
            assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= tol, (dt, b)
    ps, _ = odda.solve(prob, "lu")
    qref = odda.cross_sections(prob, ps)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-7, maxit=3000)
    assert all(r["converged"] == 1 for r in reps)
    q, _ = ctx.dda_cross_sections(p)
    for b in range(ctx.nrhs):
        for i, key in enumerate(("Qext", "Qabs")):
            assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (key, b)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_cross_sections(p, [(0.5, 0.0)])
    assert ei.value.status == D.DDA_EUNSUPPORTED


def test_periodic_slab_absorption_against_fresnel(D):
    """16 dipole layers of an infinite slab (periods 1 x 1), normal incidence, gamma = 0.01: the absorbed
    fraction per unit area matches the continuum film of the same thickness within the discretization
    error."""
    nl, m, kd = 16, 1.5 + 0.1j, 0.05
    ijk = np.stack([np.arange(nl), np.zeros(nl, int), np.zeros(nl, int)], 1)
    ctx = D.Context(0)
    ctx.dda_setup_target(ijk)
    ctx.dda_set_periodicity(1.0, 1.0, 0.01)
    ctx.dda_set_incident(kd, [(0, 0, 0)], [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("LATTDR", m)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="C128", tol=1e-10, maxit=3000)
    q, _ = ctx.dda_cross_sections(p)
    _, aeff = ctx.dda_kd_from_x(1.0)
    fres = oper.slab_fresnel_absorption(m, kd, nl)
    for b in range(2):
        absorbed = q[b, 1] * math.pi * aeff ** 2
        assert absorbed == pytest.approx(fres, rel=0.01), (b, absorbed, fres)
    # oblique incidence with a direction the replicas' phases must follow: a periodic context refuses
    # RHS of different incident directions
    ctx.dda_set_incident(kd, [(0, 0, 0), (0, 0.3, 0)], [[0, 0], [1, 0], [0, 0]], 2)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_build_green_fft()
    assert ei.value.status == D.DDA_EUNSUPPORTED


def _periodic_ctx(D, t, periods, gamma, ori, kd, m):
    ctx = D.Context(0)
    ctx.dda_setup_target(t.ijk, origin=t.origin)
    ctx.dda_set_periodicity(periods[0], periods[1], gamma)
    ctx.dda_set_incident(kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("GKDLDR", m)
    return ctx


@pytest.mark.parametrize("ori,periods", [((0.0, 0.0, 0.0), (8.0, 8.0)), ((0.3, 0.5, 0.7), (8.0, 7.0))],
                         ids=["normal", "oblique"])
def test_diffraction_orders_match_oracle(D, ori, periods):
    """A doubly periodic array of small ellipsoids with several propagating orders (kd = 1): order
    directions, the generalized Mueller matrix S^(2d)(M, N) in transmission and reflection and the
    transmission / reflection coefficients against the oracle (its LU solution, the GPU's solved to
    1e-10); the coefficients over every allowed order plus the GPU's own absorbed fraction make 1;
    a non-propagating order and a finite target are refused."""
    t = o_targets.make_target("ELLIPSOID", (3, 4, 3))
    gamma, kd, m = 0.005, 1.0, 1.4 + 0.05j
    prob = odda.build_problem(None, None, m, None, "GKDLDR", [ori], target=t, kd=kd, iorth=2, periods=periods,
                              gamma=gamma)
    ps, _ = odda.solve(prob, "lu")
    ctx = _periodic_ctx(D, t, periods, gamma, [ori], kd, m)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, solver="BICGSTAB", precision="C128", tol=1e-10, maxit=3000)
    assert all(r["converged"] == 1 for r in reps)
    k0 = prob.rhs[0].k_tf
    spec = [(M, N) for M in range(-2, 3) for N in range(-2, 3) if oper.order_direction(k0, periods, M, N) is not None]
    assert len(spec) >= 4
    dirs, mu, tr = ctx.dda_periodic_scattering(p, spec)
    q, _ = ctx.dda_cross_sections(p)
    _, aeff = ctx.dda_kd_from_x(1.0)
    pn = p.cpu().numpy()
    for s, (M, N) in enumerate(spec):
        for side, sign in enumerate((1, -1)):
            n = oper.order_direction(k0, periods, M, N, sign=sign)
            assert np.abs(dirs[s, side] - n).max() < 1e-13
            ref = oper.mueller_in_order(prob, 0, ps, n)
            assert np.abs(mu[0, s, side] - ref).max() <= 1e-6 * np.abs(ref).max(), (M, N, side)
        for b in range(2):
            ref_tr = oper.transmission_reflection(prob, b, ps[b], M, N)
            np.testing.assert_allclose(tr[b, s], ref_tr, rtol=1e-6, atol=1e-12)
    n0x = abs(k0[0]) / kd
    for b in range(2):
        absorbed = q[b, 1] * math.pi * aeff ** 2 / (periods[0] * periods[1] * n0x)
        assert tr[b].sum() + absorbed == pytest.approx(1.0, abs=1e-5)
    M_bad = int(np.ceil(2 * periods[0] / (2 * np.pi) * kd)) + 2
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_periodic_scattering(p, [(M_bad, 0)])
    assert ei.value.status == D.DDA_EINVAL
    fin = D.Context(0)
    fin.dda_setup_target(t.ijk, origin=t.origin)
    fin.dda_set_incident(kd, [ori], [[0, 0], [1, 0], [0, 0]], 2)
    fin.dda_build_green_fft()
    fin.dda_set_polarizability("GKDLDR", m)
    with pytest.raises(D.DDAError) as ei:
        fin.dda_periodic_scattering(p, [(0, 0)])
    assert ei.value.status == D.DDA_EUNSUPPORTED


@pytest.mark.parametrize("periods", [(8.0, 0.0), (0.0, 7.0)], ids=["axis_y", "axis_z"])
def test_scattering_cones_match_oracle(D, periods):
    """A target periodic along one axis: cone directions and S^(1d)(M, zeta) against the oracle on
    every allowed cone at several azimuths, and the cone-integrated power against the GPU's own
    C_sca per unit length (the oracle's energy pin, on the GPU's numbers)."""
    t = o_targets.make_target("ELLIPSOID", (3, 4, 3))
    gamma, kd, m, ori = 0.000625, 1.0, 1.4 + 0.05j, (0.2, 0.6, 0.3)
    prob = odda.build_problem(None, None, m, None, "GKDLDR", [ori], target=t, kd=kd, iorth=2, periods=periods,
                              gamma=gamma)
    ps, _ = odda.solve(prob, "lu")
    ctx = _periodic_ctx(D, t, periods, gamma, [ori], kd, m)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, solver="BICGSTAB", precision="C128", tol=1e-10, maxit=3000)
    assert all(r["converged"] == 1 for r in reps)
    k0 = prob.rhs[0].k_tf
    cones = [M for M in range(-3, 4) if oper.order_direction(k0, periods, M) is not None]
    nz = 120
    zetas = np.arange(nz) * 2 * np.pi / nz
    spec = [(M, z) for M in cones for z in zetas]
    dirs, mu, tr = ctx.dda_periodic_scattering(p, spec)
    assert tr is None
    axis = 1 if periods[0] else 2
    tot = 0.0
    for s, (M, z) in enumerate(spec):
        n = oper.order_direction(k0, periods, M, zeta=z)
        assert np.abs(dirs[s, 0] - n).max() < 1e-13 and not dirs[s, 1].any()
        if s % 17 == 0:
            ref = oper.mueller_in_order(prob, 0, ps, n)
            assert np.abs(mu[0, s, 0] - ref).max() <= 1e-6 * np.abs(ref).max(), (M, z)
        tot += mu[0, s, 0, 0, 0] * np.sqrt(1.0 - n[axis] ** 2) / kd * (2 * np.pi / nz)
    q, _ = ctx.dda_cross_sections(p)
    _, aeff = ctx.dda_kd_from_x(1.0)
    length = periods[0] or periods[1]
    csca = np.mean([(q[b, 0] - q[b, 1]) * math.pi * aeff ** 2 for b in range(2)]) / length
    assert tot == pytest.approx(csca, rel=1e-4)


def test_near_field_of_periodic_targets_matches_oracle(D):
    """DDfield for periodic targets (the replicas' dipoles with their Bloch phases and the cutoff on
    each term): E and B against the oracle at points inside, near and away from an infinite slab
    (normal incidence) and a doubly periodic array (oblique incidence); behind the slab |E|^2 is
    the (0, 0) transmission coefficient the library reports."""
    from oracle import nearfield as onf
    nl, m, kd, gamma = 8, 1.5 + 0.1j, 0.2, 0.04
    ijk = np.stack([np.arange(nl), np.zeros(nl, int), np.zeros(nl, int)], 1)
    tt = o_targets.Target(ijk=ijk, box=(nl, 1, 1), origin=np.zeros(3), a1=np.array([1.0, 0, 0]),
                          a2=np.array([0, 1.0, 0]))
    cases = [
        (tt, (1.0, 1.0), gamma, (0.0, 0.0, 0.0), kd, m, "LATTDR",
         np.array([[-15.0, 0.3, 0.2], [25.0, 0.1, 0.7], [3.5, 0.5, 0.5], [0.2, 0.1, 0.0]])),
        (o_targets.make_target("ELLIPSOID", (3, 4, 3)), (8.0, 7.0), 0.005, (0.3, 0.5, 0.7), 1.0, 1.4 + 0.05j, "GKDLDR",
         np.array([[-6.0, 1.0, 2.0], [0.3, 4.0, 3.5], [7.0, -2.0, 1.0]])),
    ]
    for t, periods, gam, ori, k, mm, presc, pts in cases:
        prob = odda.build_problem(None, None, mm, None, presc, [ori], target=t, kd=k, iorth=2, periods=periods,
                                  gamma=gam)
        ps, _ = odda.solve(prob, "lu")
        ctx = D.Context(0)
        ctx.dda_setup_target(t.ijk, origin=t.origin)
        ctx.dda_set_periodicity(periods[0], periods[1], gam)
        ctx.dda_set_incident(k, [ori], [[0, 0], [1, 0], [0, 0]], 2)
        ctx.dda_build_green_fft()
        ctx.dda_set_polarizability(presc, mm)
        p = torch.from_numpy(np.ascontiguousarray(np.stack(ps))).cuda()
        E, B = ctx.dda_near_field(p, pts)
        for b in range(2):
            rh = prob.rhs[b]
            Er, Br = onf.fields_at(pts, k, t.r, ps[b], rh.k_tf, rh.e_tf, periods=periods, gamma=gam)
            for i in range(len(pts)):
                assert np.linalg.norm(E[b, i] - Er[i]) <= 1e-9 * np.linalg.norm(Er[i]), (periods, b, i)
                assert np.linalg.norm(B[b, i] - Br[i]) <= 1e-9 * np.linalg.norm(Br[i]), (periods, b, i)
        if periods == (1.0, 1.0):
            _, _, tr = ctx.dda_periodic_scattering(p, [(0, 0)], mueller=False, tr=True)
            for b in range(2):
                assert abs(np.vdot(E[b, 1], E[b, 1]).real - tr[b, 0, 0]) <= 4e-3 * tr[b, 0, 0]

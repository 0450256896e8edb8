"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (written in each test):
  A P      relative L2 <= 1e-12 (complex128) and <= 1e-5 (complex64) against the
           oracle's direct O(N^2) sum (small targets) or its direct rows
           (sampled sites of full-size targets);
  Q_*      <= 1e-4 relative against the oracle solved to 1e-10;
  integers (sites) bit-exact (tests/test_abi_cpu.py).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import dda as odda
from oracle import targets as o_targets  # noqa: E402
from oracle import interaction as oint  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


def _oracle_problem(w, kd=None, pad=None):
    return odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations, e01_lf=w.e01,
                              iorth=w.iorth, pad=pad if pad is not None else w.pad)


def _ctx(D, w, pad=None):
    ctx = D.Context(0)
    D.setup_workload(ctx, w, pad)
    return ctx


def _rand_p(n_rhs, n, seed, dtype):
    p = W.seeded_vector((n_rhs, 3, n), seed)
    return torch.from_numpy(p).to(dtype).cuda()


SMALL = [
    W.Workload("sph12", "ELLIPSOID", (12, 12, 12), 1.33 + 0.01j, 1.0, "LATTDR", W.IDENTITY),
    W.Workload("ell_odd", "ELLIPSOID", (7, 5, 9), 1.5 + 0.1j, 2.0, "GKDLDR", W.uniform_orientations(2, 11)),
    W.Workload("cyl", "CYLINDER1", (9, 6, 2), 1.7 + 0.3j, 3.0, "CM", W.uniform_orientations(2, 12)),
    W.Workload("hex", "HEX_PRISM", (5, 10, 3), 1.33 + 0.001j, 2.5, "GKDLDR", W.uniform_orientations(1, 13)),
    W.Workload("blk", "RCTGLPRSM", (3, 17, 4), 2.0 + 1.0j, 1.5, "LATTDR", W.uniform_orientations(2, 14)),
]


@pytest.mark.parametrize("w", SMALL, ids=[w.name for w in SMALL])
def test_matvec_matches_direct_sum(D, w):
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    assert ctx.n == prob.target.n
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 3, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
            assert err <= tol, (w.name, dt, b, err)


FAST_PADS = [
    # (workload, pad): plane pair (32, 48); 5-pass with a 16-point x length (one-stage pass A);
    # plane (40, 40); 5-pass c64 and c128 with odd boxes and ragged y tiles
    (W.Workload("ell_p1", "ELLIPSOID", (12, 16, 24), 1.5 + 0.1j, 2.0, "GKDLDR", W.uniform_orientations(1, 41)),
     (24, 32, 48)),
    (W.Workload("blk_p2", "RCTGLPRSM", (3, 17, 4), 2.0 + 1.0j, 1.5, "LATTDR", W.uniform_orientations(2, 42)),
     (16, 40, 40)),
    (W.Workload("cyl_p3", "CYLINDER1", (30, 20, 1), 1.33 + 0.05j, 3.0, "CM", W.uniform_orientations(1, 43)),
     (64, 40, 40)),
    (W.Workload("ell_p4", "ELLIPSOID", (11, 13, 6), 1.4 + 0.2j, 2.0, "GKDLDR", W.uniform_orientations(2, 44)),
     (24, 32, 16)),
    # plane pair (32, 32) with an odd ny*nz = 15*15: the plane pass without bulk-copy staging
    (W.Workload("ell_p5", "ELLIPSOID", (10, 15, 15), 1.5 + 0.05j, 2.0, "LATTDR", W.uniform_orientations(1, 45)),
     (24, 32, 32)),
]


@pytest.mark.parametrize("w,pad", FAST_PADS, ids=[w.name for w, _ in FAST_PADS])
def test_matvec_fast_kernels_match_direct_sum(D, w, pad):
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 8, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
            assert err <= tol, (w.name, dt, b, err)


@pytest.mark.parametrize("w,pad", FAST_PADS, ids=[w.name for w, _ in FAST_PADS])
def test_double_float_product_matches_direct_sum(D, w, pad):
    """complex128 vectors, double-float arithmetic (DDA_C128DF): within 1e-12 of the oracle's
    direct sum and of the complex128 product (48-bit significands, error ~1e-13 of |A P|)."""
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    p = _rand_p(ctx.nrhs, ctx.n, 8, torch.complex128)
    ap_df = torch.empty_like(p)
    ap_64 = torch.empty_like(p)
    ctx.dda_matvec(p, ap_df, double_float=True)
    ctx.dda_matvec(p, ap_64)
    torch.cuda.synchronize()
    pn = p.cpu().numpy()
    got = ap_df.cpu().numpy()
    fp64 = ap_64.cpu().numpy()
    for b in range(ctx.nrhs):
        ref = odda.apply_a(prob, b, pn[b], "direct")
        assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= 1e-12, (w.name, b)
        assert np.linalg.norm(got[b] - fp64[b]) / np.linalg.norm(fp64[b]) <= 1e-12, (w.name, b)


def test_double_float_product_needs_compile_time_schedule(D, monkeypatch):
    monkeypatch.setenv("DDA_SCHEDULE", "generic")
    w, pad = FAST_PADS[0]
    ctx = _ctx(D, w, pad)
    p = _rand_p(ctx.nrhs, ctx.n, 8, torch.complex128)
    with pytest.raises(D.DDAError, match="DDA_EUNSUPPORTED"):
        ctx.dda_matvec(p, torch.empty_like(p), double_float=True)
    # the solve still runs: its true residuals fall back to the complex128 product
    p = torch.zeros_like(p)
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-6, maxit=500)
    assert all(r["converged"] for r in reps)


def test_double_float_true_residuals_are_fp64_accurate(D):
    """A mixed solve to 1e-8 takes its true residuals from the double-float product; the residual it
    reports matches |E - A P| / |E| recomputed with the complex128 product."""
    w = W.ELLIPSOID64
    ctx = _ctx(D, w)
    assert D.dda_schedule_info(ctx, D.DDA_C128)[:2] == (5, 1)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-8, maxit=3000)
    e = torch.empty_like(p)
    ctx.dda_incident_field(e)
    ap = torch.empty_like(p)
    ctx.dda_matvec(p, ap)
    torch.cuda.synchronize()
    for b, r in enumerate(reps):
        rel = float(torch.linalg.vector_norm(e[b] - ap[b]) / torch.linalg.vector_norm(e[b]))
        assert r["converged"] == 1 and rel <= 1e-8, (b, rel)
        assert abs(r["true_rel_resid"] - rel) <= 1e-11, (b, r["true_rel_resid"], rel)


@pytest.mark.parametrize("sched", ["cluster2", "cluster4"])
@pytest.mark.parametrize("w,pad", FAST_PADS[:3], ids=[w.name for w, _ in FAST_PADS[:3]])
def test_cluster_plane_matches_direct_sum(D, monkeypatch, w, pad, sched):
    """The plane pass split over a thread-block cluster, on plane pairs (32, 48) and (40, 40)
    with odd and ragged boxes (pass-A rows shared unevenly between the CTAs)."""
    monkeypatch.setenv("DDA_SCHEDULE", sched)
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    p = _rand_p(ctx.nrhs, ctx.n, 18, torch.complex64)
    ap = torch.empty_like(p)
    ctx.dda_matvec(p, ap)
    torch.cuda.synchronize()
    info = D.dda_schedule_info(ctx, D.DDA_C64)
    assert info[0] == 3 and info[4] == int(sched[-1]), info
    pn = p.cpu().numpy().astype(np.complex128)
    got = ap.cpu().numpy().astype(np.complex128)
    for b in range(ctx.nrhs):
        ref = odda.apply_a(prob, b, pn[b], "direct")
        err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (w.name, sched, b, err)


@pytest.mark.parametrize("w,pad", FAST_PADS, ids=[w.name for w, _ in FAST_PADS])
def test_bulk_staged_plane_matches_direct_sum(D, monkeypatch, w, pad):
    """The plane pass with its HBM blocks staged by bulk copies (where the grid allows it)."""
    monkeypatch.setenv("DDA_BULK", "1")
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    p = _rand_p(ctx.nrhs, ctx.n, 23, torch.complex64)
    ap = torch.empty_like(p)
    ctx.dda_matvec(p, ap)
    torch.cuda.synchronize()
    pn = p.cpu().numpy().astype(np.complex128)
    got = ap.cpu().numpy().astype(np.complex128)
    for b in range(ctx.nrhs):
        ref = odda.apply_a(prob, b, pn[b], "direct")
        err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (w.name, b, err)


@pytest.mark.parametrize("w,pad", FAST_PADS, ids=[w.name for w, _ in FAST_PADS])
def test_x_one_component_per_cta_matches_direct_sum(D, monkeypatch, w, pad):
    """The x passes with one field component per CTA, both precisions."""
    monkeypatch.setenv("DDA_XCOMP", "1")
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    assert D.dda_schedule_info(ctx, D.DDA_C64)[7] in (0, 1)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 29, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
            assert err <= tol, (w.name, dt, b, err)


@pytest.mark.parametrize("xtile", ["4", "8"])
@pytest.mark.parametrize("w,pad", FAST_PADS, ids=[w.name for w, _ in FAST_PADS])
def test_x_tile_heights_match_direct_sum(D, monkeypatch, w, pad, xtile):
    """The x passes with short tiles (4 or 8 y rows per CTA), both precisions, ragged y tiles."""
    monkeypatch.setenv("DDA_XTILE", xtile)
    ctx = _ctx(D, w, pad)
    prob = _oracle_problem(w)
    info = D.dda_schedule_info(ctx, D.DDA_C64)
    if info[1]:
        assert info[5] == int(xtile), info
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 19, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            err = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
            assert err <= tol, (w.name, xtile, dt, b, err)


def test_bounded_bulk_wait_gives_up_and_device_stays_usable(D):
    """The bounded wait of the bulk-copy path ends by itself on a barrier that never completes
    (no fault, no hang), and the device keeps working afterwards."""
    assert D.dda_selftest_bulk_wait(0) is True
    w = FAST_PADS[0][0]
    ctx = _ctx(D, w, FAST_PADS[0][1])
    p = _rand_p(ctx.nrhs, ctx.n, 3, torch.complex64)
    ap = torch.empty_like(p)
    ctx.dda_matvec(p, ap)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(ap)).all()


def test_fast_and_generic_engines_agree(D, monkeypatch):
    w = W.ELLIPSOID64
    out = {}
    for mode in ("default", "generic"):
        if mode == "generic":
            monkeypatch.setenv("DDA_SCHEDULE", "generic")
        ctx = _ctx(D, w)
        p = _rand_p(ctx.nrhs, ctx.n, 9, torch.complex64)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        out[mode] = ap.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(out["default"] - out["generic"]) / np.linalg.norm(out["generic"])
    assert err <= 2e-6, err


@pytest.mark.parametrize("sched", ["generic", "fast5", "plane512", "plane768", "cluster2", "cluster4", "bulk", None])
def test_every_schedule_matches_direct_rows(D, monkeypatch, sched):
    """Each launch schedule the autotuner can pick, pinned through DDA_SCHEDULE, on the 64x48x32 grid."""
    if sched == "bulk":
        monkeypatch.setenv("DDA_BULK", "1")
    elif sched:
        monkeypatch.setenv("DDA_SCHEDULE", sched)
    w = W.ELLIPSOID64
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    rows = np.sort(np.random.default_rng(7).choice(ctx.n, 16, replace=False))
    for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
        p = _rand_p(ctx.nrhs, ctx.n, 10, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        info = D.dda_schedule_info(ctx, D.DDA_C64 if dt == torch.complex64 else D.DDA_C128)
        if sched == "fast5":
            assert info[0] == 5 and info[1] == 1
        if sched in ("plane512", "plane768") and dt == torch.complex64:
            assert info[0] == 3 and info[2] == int(sched[-3:])
        if sched in ("cluster2", "cluster4") and dt == torch.complex64:
            assert info[0] == 3 and info[4] == int(sched[-1])
        if sched == "bulk" and dt == torch.complex64:
            assert info[0] == 3 and info[6] == 1
        for b in range(ctx.nrhs):
            pb = p[b].cpu().numpy().astype(np.complex128)
            ref = oint.matvec_direct(prob.target.r, prob.kd, prob.rhs[b].inv_alpha, pb, rows=rows)
            got = ap[b].cpu().numpy().astype(np.complex128)[:, rows]
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (sched, dt, b, err)


@pytest.mark.parametrize("zfuse", ["1", "0"])
def test_register_fused_z_columns_match_direct_sum(D, monkeypatch, zfuse):
    """The 5-pass schedule with the z columns' middle stages fused in registers (the kernel the
    tuner may pick for long z transforms: Pz = 160 here, 320 on the hexagonal prism), pinned on and
    off, complex64 against the oracle's direct sum; complex128 products keep the default kernel."""
    monkeypatch.setenv("DDA_SCHEDULE", "fast5")
    monkeypatch.setenv("DDA_ZFUSE", zfuse)
    w = W.Workload("ell_z160", "ELLIPSOID", (14, 11, 80), 1.5 + 0.05j, 3.0, "LATTDR", W.uniform_orientations(2, 31),
                   pad=(32, 24, 160))
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    info = D.dda_schedule_info(ctx, D.DDA_C64)
    assert info[0] == 5 and info[8] == int(zfuse), info
    rows = np.concatenate([[0, ctx.n - 1], np.sort(np.random.default_rng(3).choice(ctx.n, 40, replace=False))])
    for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
        p = _rand_p(ctx.nrhs, ctx.n, 17, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        for b in range(ctx.nrhs):
            pb = p[b].cpu().numpy().astype(np.complex128)
            ref = oint.matvec_direct(prob.target.r, prob.kd, prob.rhs[b].inv_alpha, pb, rows=rows)
            got = ap[b].cpu().numpy().astype(np.complex128)[:, rows]
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, (zfuse, dt, b)


def test_matvec_nondefault_pad_and_tail_tiles(D):
    # odd box sizes against a padded grid larger than 2N (pruned FFT inputs shorter than L/2)
    w = W.Workload("ell_pad", "ELLIPSOID", (11, 13, 6), 1.4 + 0.2j, 2.0, "GKDLDR", W.uniform_orientations(1, 21),
                   pad=(30, 30, 16))
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    p = _rand_p(ctx.nrhs, ctx.n, 4, torch.complex128)
    ap = torch.empty_like(p)
    ctx.dda_matvec(p, ap)
    got = ap.cpu().numpy()
    for b in range(ctx.nrhs):
        ref = odda.apply_a(prob, b, p.cpu().numpy()[b], "direct")
        assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("w", [W.ELLIPSOID64, W.PRISM48], ids=["ellipsoid64", "prism48_b128"])
def test_matvec_full_size_sampled_rows(D, w):
    """Full-size grids in the launch configuration the benchmark times (all RHS in one batch)."""
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(ctx.n, 24, replace=False))
    rows = np.concatenate([[0, ctx.n - 1], rows])
    rhs = [0, ctx.nrhs - 1]
    for dt, tol, dfl in ((torch.complex64, 1e-5, False), (torch.complex128, 1e-12, False),
                         (torch.complex128, 1e-12, True)):
        p = _rand_p(ctx.nrhs, ctx.n, 6, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap, double_float=dfl)
        torch.cuda.synchronize()
        for b in rhs:
            pb = p[b].cpu().numpy().astype(np.complex128)
            ref = oint.matvec_direct(prob.target.r, prob.kd, prob.rhs[b].inv_alpha, pb, rows=rows)
            got = ap[b].cpu().numpy().astype(np.complex128)[:, rows]
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (dt, dfl, b, err)


def test_matvec_large_hexprism_sampled_rows(D):
    """The 1.69M-dipole hexagonal prism on its 256x256x320 grid, all 32 RHS in one batch."""
    w = W.HEXPRISM160
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    assert ctx.n == prob.target.n
    rng = np.random.default_rng(9)
    rows = np.concatenate([[0, ctx.n - 1], rng.choice(ctx.n, 4, replace=False)])
    for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
        p = _rand_p(ctx.nrhs, ctx.n, 12, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        for b in (0, ctx.nrhs - 1):
            pb = p[b].cpu().numpy().astype(np.complex128)
            ref = oint.matvec_direct(prob.target.r, prob.kd, prob.rhs[b].inv_alpha, pb, rows=rows, chunk=2)
            got = ap[b].cpu().numpy().astype(np.complex128)[:, rows]
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (dt, b, err)
        del p, ap
        torch.cuda.empty_cache()


def test_incident_field_matches_oracle(D):
    w = SMALL[1]
    ctx = _ctx(D, w)
    prob = _oracle_problem(w)
    e = torch.empty((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.dda_incident_field(e)
    got = e.cpu().numpy()
    for b in range(ctx.nrhs):
        np.testing.assert_allclose(got[b], prob.rhs[b].e_inc, rtol=0, atol=1e-13)


def _oracle_q(w, tol=1e-10):
    prob = _oracle_problem(w)
    method = "lu" if prob.target.n * 3 <= 3000 else "bicgstab"
    ps, _ = odda.solve(prob, method, tol=tol, workers=-1)
    return prob, ps, odda.cross_sections(prob, ps)


@pytest.mark.parametrize("solver,precision", [("BICGSTAB", "C128"), ("BICGSTAB", "MIXED"), ("BICGSTAB", "C64"),
                                              ("CCG", "C128"), ("CCG", "MIXED"), ("BICGSTAB2", "C128"),
                                              ("BICGSTAB2", "MIXED"), ("BICGSTAB2", "C64")])
def test_solve_sphere12_cross_sections(D, solver, precision):
    w = W.SPHERE12
    prob, ps, qref = _oracle_q(w)
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, st = ctx.dda_solve(p, solver=solver, precision=precision, tol=1e-5, maxit=2000, normal_eq=True)
    for r in reps:
        assert r["converged"] == 1 and r["true_rel_resid"] <= 1e-5
        assert r["normal_eq_ratio"] <= 1e-4
    # the reported normal-equation ratio (guide, "Error Tolerance") against the oracle's FP64 value for
    # the same GPU solution, with the oracle's dense A: same quantity, so agreement to rounding
    got_p = p.cpu().numpy()
    from oracle import solvers as osol
    for b in range(ctx.nrhs):
        a = oint.dense_matrix(prob.target.r, prob.kd, prob.rhs[b].inv_alpha)
        ref = osol.normal_eq_ratio(lambda v: a @ v, got_p[b].reshape(-1), prob.rhs[b].e_inc.reshape(-1))
        assert reps[b]["normal_eq_ratio"] == pytest.approx(ref, rel=1e-6), (b, reps[b]["normal_eq_ratio"], ref)
        tr = np.linalg.norm(prob.rhs[b].e_inc.reshape(-1) - a @ got_p[b].reshape(-1)) / np.linalg.norm(
            prob.rhs[b].e_inc)
        assert abs(reps[b]["true_rel_resid"] - tr) <= 1e-10, (b, reps[b]["true_rel_resid"], tr)
    q, _ = ctx.dda_cross_sections(p)
    for b in range(ctx.nrhs):
        for i, key in enumerate(("Qext", "Qabs", "Qsca")):
            assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (key, b)
        assert abs(q[b, 3] - qref[b]["Qpha"]) <= 1e-4 * abs(qref[b]["Qext"]), b


def test_solve_ellipsoid64_mixed_vs_oracle(D):
    w = W.ELLIPSOID64
    prob, ps, qref = _oracle_q(w, tol=1e-10)
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=1000)
    assert all(r["converged"] for r in reps)
    q, _ = ctx.dda_cross_sections(p)
    for b in range(ctx.nrhs):
        for i, key in enumerate(("Qext", "Qabs", "Qsca")):
            assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (key, b)
        assert abs(q[b, 3] - qref[b]["Qpha"]) <= 1e-4 * abs(qref[b]["Qext"]), b
    # the solution itself: relative L2 against the oracle's
    got = p.cpu().numpy()
    for b in range(ctx.nrhs):
        assert np.linalg.norm(got[b] - ps[b]) / np.linalg.norm(ps[b]) < 1e-4


def test_mueller_matches_oracle(D):
    w = W.Workload("ell_m", "ELLIPSOID", (8, 6, 5), 1.5 + 0.1j, 2.0, "GKDLDR", W.uniform_orientations(2, 31))
    prob, ps, qref = _oracle_q(w)
    ctx = _ctx(D, w)
    p = torch.from_numpy(np.stack(ps)).cuda()
    dirs = [(0.0, 0.0), (0.7, 0.3), (math.pi / 2, 1.1), (2.5, 4.0), (math.pi, 0.0)]
    q, mm = ctx.dda_cross_sections(p, dirs)
    for o in range(2):
        ref = odda.mueller(prob, ps, dirs, ori_index=o)
        np.testing.assert_allclose(mm[o], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    for b in range(ctx.nrhs):
        assert q[b, 0] == pytest.approx(qref[b]["Qext"], rel=1e-12)
        assert q[b, 1] == pytest.approx(qref[b]["Qabs"], rel=1e-12)


def test_worked_example_au_block_on_gpu(D):
    """The guide's printed sample calculation, solved by the GPU path."""
    from conftest import load_golden
    g, rows = load_golden("au_block_worked_example.txt")
    w = W.AU_BLOCK
    ctx = _ctx(D, w)
    assert ctx.n == int(g["NAT0"])
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=2000)
    assert all(r["converged"] for r in reps)
    dirs = [(math.radians(r[0]), math.radians(r[1])) for r in rows]
    q, mm = ctx.dda_cross_sections(p, dirs)
    for b in range(2):
        assert q[b, 0] == pytest.approx(g["Qext"], rel=1e-4)
        assert q[b, 1] == pytest.approx(g["Qabs"], rel=1e-4)
        assert q[b, 2] == pytest.approx(g["Qsca"], rel=1e-4)
        assert q[b, 3] == pytest.approx(g["Qpha"], rel=2e-4)
    for r, m in zip(rows, mm[0]):
        assert m[0, 0] == pytest.approx(r[2], rel=5e-4)
    # backscattering efficiency Q_bk = (dC_sca/dOmega at theta = pi) / (pi a_eff^2) = S11(pi) / (pi (k a_eff)^2)
    back = [m for r, m in zip(rows, mm[0]) if r[0] == 180.0]
    assert len(back) == 1
    ka = ctx.kd * (3.0 * ctx.n / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert back[0][0, 0] / (math.pi * ka ** 2) == pytest.approx(g["Qbk"], rel=6e-4)  # printed values agree to 3e-5


def test_bicgstab2_follows_the_oracle(D):
    """GPU BiCGstab(2) in complex128 against the oracle's BiCGstab(l = 2) on the same system: same
    cycle count to the same tolerance (up to one cycle of rounding drift) and the same solution."""
    from oracle import solvers as osol
    w = W.SPHERE12
    prob = _oracle_problem(w)
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, solver="BICGSTAB2", precision="C128", tol=1e-8, maxit=2000, check_every=1)
    got = p.cpu().numpy()
    for b in range(ctx.nrhs):
        rh = prob.rhs[b]
        shape = rh.e_inc.shape

        def op(v, b=b):
            return odda.apply_a(prob, b, v.reshape(shape), "direct").reshape(-1)
        x, it, _ = osol.bicgstab_l(op, rh.e_inc.reshape(-1), ell=2, tol=1e-8)
        assert reps[b]["converged"] == 1 and reps[b]["true_rel_resid"] <= 1e-8
        assert abs(reps[b]["iters"] - it) <= 2, (reps[b]["iters"], it)
        xs = x.reshape(shape)
        assert np.linalg.norm(got[b] - xs) / np.linalg.norm(xs) < 1e-6


def test_worked_example_au_block_bicgstab2(D):
    """The guide's sample calculation used its BiCGstab(2)-family solver (PBCGS2): 27 and 29 iterations
    for the two polarizations at TOL = 1e-5 (its normal-equation stopping rule), read here as
    BiCGstab(2) cycles (two BiCG steps, four products each).  BiCGstab(2) here, stopping on
    |E - AP|/|E| <= 1e-5, needs a cycle count in the same range and reproduces the efficiencies."""
    from conftest import load_golden
    g, rows = load_golden("au_block_worked_example.txt")
    w = W.AU_BLOCK
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, solver="BICGSTAB2", precision="MIXED", tol=1e-5, maxit=2000, normal_eq=True)
    its = [r["iters"] for r in reps]
    print("BiCGstab(2) iterations on the Au block:", its, "normal-equation ratios",
          [r["normal_eq_ratio"] for r in reps])
    assert all(r["converged"] for r in reps)
    cycles = [i // 2 for i in its]
    assert all(20 <= c <= 40 for c in cycles), cycles
    q, _ = ctx.dda_cross_sections(p)
    for b in range(2):
        assert q[b, 0] == pytest.approx(g["Qext"], rel=1e-4)
        assert q[b, 1] == pytest.approx(g["Qabs"], rel=1e-4)
        assert q[b, 2] == pytest.approx(g["Qsca"], rel=1e-4)


def test_angular_averages_match_oracle(D):
    """Q_sca by angular integration, <cos>, <cos^2> and the g vector over the guide's direction set,
    GPU far-field sums against the oracle's direct evaluation, several orientations and two eta."""
    from oracle import observables as oobs
    w = W.Workload("ell_ang", "ELLIPSOID", (8, 6, 5), 1.5 + 0.1j, 2.0, "GKDLDR", W.uniform_orientations(2, 51))
    prob, ps, qref = _oracle_q(w)
    ctx = _ctx(D, w)
    p = torch.from_numpy(np.stack(ps)).cuda()
    geo = math.pi * prob.target.aeff ** 2
    for eta in (0.5, 0.2):
        out, nd = ctx.dda_angular_averages(p, eta)
        for b in range(ctx.nrhs):
            c_int, g1, g2, gv, ndir = oobs.angular_averages(prob.kd, prob.target.r, ps[b], prob.rhs[b].axes, prob.x, eta)
            assert nd == ndir
            assert out[b, 0] == pytest.approx(c_int / geo, rel=1e-5), (eta, b)
            assert abs(out[b, 1] - g1) <= 1e-5 and abs(out[b, 2] - g2) <= 1e-5, (eta, b)
            np.testing.assert_allclose(out[b, 3:], gv, atol=1e-5)
            # optical theorem: integrated scattering against Q_ext - Q_abs
            assert out[b, 0] == pytest.approx(qref[b]["Qsca"], rel=2e-2)


def test_angular_averages_au_block(D):
    """The guide's sample calculation: N_sca = 2292 directions at eta = 0.5, where <cos theta> is 0.4563
    (the oracle's value with the same direction set) and Q_sca by integration is 2 % above
    Q_ext - Q_abs; with finer sampling (eta = 0.1) both converge to the printed 0.46029 and 2.4287."""
    from conftest import load_golden
    g, _ = load_golden("au_block_worked_example.txt")
    w = W.AU_BLOCK
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=2000)
    out, nd = ctx.dda_angular_averages(p, 0.5)
    print("Au block angular averages (Qsca_int, <cos>, <cos^2>):", out[:, :3].tolist(), "N_sca", nd)
    assert nd == 2292
    for b in range(2):
        assert out[b, 0] == pytest.approx(g["Qsca"], rel=3e-2)
        assert abs(out[b, 1] - 0.4563) < 2e-3
    fine, nd_fine = ctx.dda_angular_averages(p, 0.1)
    print("eta 0.1:", fine[:, :3].tolist(), "N_sca", nd_fine)
    for b in range(2):
        assert fine[b, 0] == pytest.approx(g["Qsca"], rel=5e-3)
        assert abs(fine[b, 1] - 0.46029) < 1e-3


def test_orientation_averaged_efficiencies(D):
    """Orientational averaging with the guide's (beta, Theta, Phi) sampling (Simpson in cos Theta):
    GPU batched solve over all orientations, weighted average, against the oracle's."""
    from oracle import orientation as oori
    args = ((0, 360), 2, (0, 180), 3, (0, 360), 2)
    ori, wts = D.dda_orientation_grid(*args)
    w = W.Workload("ell_avg", "ELLIPSOID", (8, 6, 5), 1.5 + 0.1j, 2.0, "GKDLDR", tuple(map(tuple, ori)))
    ref_ori, ref_w = oori.orientation_grid(*args)
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, ref_ori)
    ps, _ = odda.solve(prob, "lu")
    qref = odda.cross_sections(prob, ps)
    qr = np.array([[q["Qext"], q["Qabs"], q["Qsca"]] for q in qref])
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-6, maxit=2000)
    q, _ = ctx.dda_cross_sections(p)
    avg = D.orientation_average(q[:, :3], wts)
    avg_ref = D.orientation_average(qr, ref_w)
    np.testing.assert_allclose(avg, avg_ref, rtol=2e-5)
    # the average differs from any single orientation (the ellipsoid is not isotropic)
    assert np.ptp(q[:, 0]) > 1e-3 * avg[0, 0]


@pytest.mark.parametrize("aniso", [False, True])
def test_multi_composition_targets(D, aniso):
    """Site-list targets of several materials, isotropic (one composition per site) or anisotropic
    (one per site and axis, the guide's FROM_FILE compositions): product, solve and efficiencies
    against the oracle."""
    t = o_targets.make_target("ELLIPSOID", (9, 7, 6))
    if aniso:
        comp = np.stack([t.ijk[:, 2] % 2, (t.ijk[:, 0] // 3) % 3, np.full(t.n, 1)], axis=1)
    else:
        comp = (t.ijk[:, 0] + t.ijk[:, 2]) % 3
    m = [1.5 + 0.1j, 1.33 + 0.01j, 2.2 + 0.6j]
    ori = W.uniform_orientations(2, 61)
    prob = odda.build_problem(None, None, m, 2.5, "GKDLDR", ori, target=t, comp=comp)
    ctx = D.Context(0)
    ctx.dda_setup_target(t.ijk, icomp=comp + 1, origin=t.origin)
    ctx.dda_set_incident(prob.kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("GKDLDR", m)
    ia = ctx.dda_get_inv_alpha()
    for b in range(ctx.nrhs):
        for mi in range(3):
            for a in range(3):
                sel = comp[:, a] == mi if aniso else comp == mi
                if np.any(sel):
                    assert ia[b, mi, a] == pytest.approx(prob.rhs[b].inv_alpha[sel, a][0], rel=1e-13)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 31, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= tol, (aniso, dt, b)
    ps, _ = odda.solve(prob, "lu")
    qref = odda.cross_sections(prob, ps)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-6, maxit=2000)
    q, _ = ctx.dda_cross_sections(p)
    for b in range(ctx.nrhs):
        for i, key in enumerate(("Qext", "Qabs", "Qsca")):
            assert q[b, i] == pytest.approx(qref[b][key], rel=1e-4), (aniso, key, b)


@pytest.mark.parametrize("sched", ["plane512", "fast5"])
def test_rows_with_gaps_and_empty_rows(D, monkeypatch, sched):
    """A site list whose box rows are single runs, several runs (holes) or empty: the x passes read
    single-run rows through their run descriptor and the others through the box map; the product
    against the oracle's direct sum on the 3-pass and the 5-pass schedules."""
    monkeypatch.setenv("DDA_SCHEDULE", sched)
    rng = np.random.default_rng(71)
    box = (11, 9, 13)
    full = np.stack(np.meshgrid(np.arange(box[0]), np.arange(box[1]), np.arange(box[2]), indexing="ij"),
                    axis=-1).reshape(-1, 3)
    keep = rng.random(len(full)) < 0.6                 # holes: most rows have several runs
    keep &= ~((full[:, 1] == 4) & (full[:, 2] % 3 == 0))  # some rows empty
    solid = (full[:, 1] == 2) | (full[:, 2] == 5)      # some rows one run
    keep |= solid & (full[:, 0] >= 2) & (full[:, 0] < 9)
    ijk = full[keep].astype(np.int32)
    ijk = ijk[rng.permutation(len(ijk))]               # any order: both sides sort x-fastest
    t = o_targets.from_sites(ijk, origin=(0.0, 0.0, 0.0))
    m = 1.5 + 0.1j
    ori = W.uniform_orientations(2, 72)
    prob = odda.build_problem(None, None, m, 2.0, "GKDLDR", ori, target=t)
    ctx = D.Context(0)
    ctx.dda_setup_target(ijk, origin=(0.0, 0.0, 0.0))
    sites, _ = ctx.dda_get_sites()
    assert np.array_equal(sites - sites.min(axis=0), t.ijk)
    ctx.dda_set_incident(prob.kd, ori, [[0, 0], [1, 0], [0, 0]], 2)
    ctx.dda_build_green_fft((24, 32, 32))   # (Py, Pz) = (32, 32): a plane pair with compile-time kernels
    ctx.dda_set_polarizability("GKDLDR", [m])
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(ctx.nrhs, ctx.n, 73, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        pn = p.cpu().numpy().astype(np.complex128)
        got = ap.cpu().numpy().astype(np.complex128)
        for b in range(ctx.nrhs):
            ref = odda.apply_a(prob, b, pn[b], "direct")
            assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= tol, (sched, dt, b)
    assert D.dda_schedule_info(ctx, D.DDA_C64)[:2] == ((3, 1) if sched == "plane512" else (5, 1))


def test_warm_start_from_solution_needs_no_iterations(D):
    w = W.SPHERE12
    prob, ps, _ = _oracle_q(w, tol=1e-12)
    ctx = _ctx(D, w)
    p = torch.from_numpy(np.stack(ps)).cuda()
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, warm_start=True)
    assert all(r["iters"] == 0 and r["converged"] for r in reps)


@pytest.mark.parametrize("w", [W.ELLIPSOID64, W.AU_BLOCK, W.PRISM48], ids=["ellipsoid64", "au_block_5pass",
                                                                       "prism48_b128"])
def test_folded_bicgstab_updates_match_separate_kernels(D, monkeypatch, w):
    """BiCGstab with its vector updates and dot products folded into the product's x passes (the
    default) against the separate vector kernels (DDA_FUSE=0): the 3-pass and 5-pass schedules and
    128 RHS in one batch, same iterations (the scalars are rounded to FP32 before use, so a different
    reduction order does not reach the iterates), same products and residuals, same efficiencies."""
    out = {}
    for fuse in ("0", "1"):
        monkeypatch.setenv("DDA_FUSE", fuse)
        ctx = _ctx(D, w)
        p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
        reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-5, maxit=3000)
        q, _ = ctx.dda_cross_sections(p)
        out[fuse] = (reps, q, p.cpu().numpy())
        del ctx
    (r0, q0, p0), (r1, q1, p1) = out["0"], out["1"]
    for a, b in zip(r0, r1):
        assert a["converged"] == 1 and b["converged"] == 1
        assert abs(a["iters"] - b["iters"]) <= 1 and abs(a["matvecs"] - b["matvecs"]) <= 2, (a, b)
        assert b["true_rel_resid"] <= 1e-5
    np.testing.assert_allclose(q1[:, :3], q0[:, :3], rtol=1e-5)
    assert np.linalg.norm(p1 - p0) / np.linalg.norm(p0) < 1e-4


def test_graph_and_plain_launches_agree(D):
    w = SMALL[1]
    ctx = _ctx(D, w)
    out = []
    for g in (True, False):
        p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
        reps, _ = ctx.dda_solve(p, precision="C128", tol=1e-8, use_graph=g)
        out.append((p.cpu().numpy(), [r["iters"] for r in reps]))
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][0], out[1][0])


def test_state_errors_on_device(D):
    ctx = D.Context(0)
    p = torch.zeros((1, 3, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_matvec(p, torch.empty_like(p), 1)
    assert ei.value.status == D.DDA_ESTATE
    ctx.dda_setup_shape("ELLIPSOID", (4, 4, 4))
    ctx.dda_set_incident(0.3, [(0, 0, 0)])
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_build_green_fft((9, 8, 8))
    assert ei.value.status == D.DDA_EINVAL


def test_solver_reports_nonconvergence(D):
    w = SMALL[2]
    ctx = _ctx(D, w)
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, st = ctx.dda_solve(p, precision="C128", tol=1e-14, maxit=3, raise_on_noconv=False)
    assert st == D.DDA_ENOCONV
    assert all(r["converged"] == 0 and r["true_rel_resid"] > 1e-14 for r in reps)


@pytest.mark.parametrize("ijk", [np.array([[0, 0, 0]]), np.stack([np.arange(7), np.zeros(7, int), np.zeros(7, int)], 1),
                                 np.array([[0, 0, 0], [3, 0, 0], [0, 2, 5]])],
                         ids=["one_dipole", "line_of_7", "three_scattered"])
def test_degenerate_targets(D, ijk):
    """Degenerate targets: a single dipole (no interactions: A = alpha^{-1}, and C_ext = 4 pi k Im(alpha)
    for real-valued field strength 1 by the optical theorem of one dipole), a one-dimensional line,
    and three isolated sites; one orientation, one polarization (iorth = 1, a single RHS).  Product
    against the direct sum and Q_ext / Q_abs against the oracle's LU solution."""
    ijk = ijk.astype(np.int32)
    t = o_targets.from_sites(ijk, origin=(0.0, 0.0, 0.0))
    m, kd = 1.5 + 0.2j, 0.4
    ori = [(0.3, 0.7, 0.2)]
    prob = odda.build_problem(None, None, m, None, "GKDLDR", ori, target=t, kd=kd, iorth=1)
    ctx = D.Context(0)
    ctx.dda_setup_target(ijk, origin=(0.0, 0.0, 0.0))
    ctx.dda_set_incident(kd, ori, [[0, 0], [1, 0], [0, 0]], 1)
    ctx.dda_build_green_fft()
    ctx.dda_set_polarizability("GKDLDR", m)
    assert ctx.nrhs == 1 and ctx.n == len(ijk)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        p = _rand_p(1, ctx.n, 91, dt)
        ap = torch.empty_like(p)
        ctx.dda_matvec(p, ap)
        torch.cuda.synchronize()
        ref = odda.apply_a(prob, 0, p.cpu().numpy()[0].astype(np.complex128), "direct")
        got = ap.cpu().numpy()[0].astype(np.complex128)
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), dt
    ps, _ = odda.solve(prob, "lu")
    qref = odda.cross_sections(prob, ps)
    p = torch.zeros((1, 3, ctx.n), dtype=torch.complex128, device="cuda")
    reps, _ = ctx.dda_solve(p, precision="MIXED", tol=1e-9, maxit=200)
    assert reps[0]["converged"] == 1
    q, _ = ctx.dda_cross_sections(p)
    assert q[0, 0] == pytest.approx(qref[0]["Qext"], rel=1e-6)
    assert q[0, 1] == pytest.approx(qref[0]["Qabs"], rel=1e-6)
    if len(ijk) == 1:
        # one dipole: P = alpha E, C_ext = 4 pi k Im(E* . alpha E) with |E| = 1 (alpha diagonal, per axis)
        rh = prob.rhs[0]
        alpha = 1.0 / rh.inv_alpha[0]
        cext = 4 * np.pi * kd * np.imag(np.sum(np.conj(rh.e_tf) * alpha * rh.e_tf))
        assert q[0, 0] * np.pi * t.aeff ** 2 == pytest.approx(cext, rel=1e-9)

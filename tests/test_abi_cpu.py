"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and
its host-side set-up (targets, incidence, polarizabilities) matches the oracle.

These run without a GPU through a host-only context (device = -1).
"""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import orientation as o_ori
from oracle import polarizability as o_pol
from oracle import targets as o_tgt
from paper_1002_1505_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    from paper_1002_1505_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1002_1505_gb300 import dda
    return dda


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "dda.h")).read()
    return sorted(set(re.findall(r"DDA_API\s+[\w\s\*]*?\b(dda_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(D):
    names = _declared_symbols()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", D.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(dda_\w+)", out))
    for nm in names:
        assert nm in exported, nm
        assert getattr(D.LIB, nm) is not None
    # nothing else leaks out of the C ABI
    assert exported == set(names)


def test_version_string(D):
    assert "sm_103a" in D.dda_version()


ALL_SHAPES = [("ELLIPSOID", (12, 12, 12)), ("ELLIPSOID", (64, 48, 32)), ("ELLIPSOID", (7, 5, 9)),
              ("RCTGLPRSM", (32, 64, 64)), ("RCTGLPRSM", (3, 5, 2)), ("CYLINDER1", (32, 16, 1)),
              ("CYLINDER1", (64, 40, 2)), ("CYLINDER1", (20, 48, 3)), ("HEX_PRISM", (160, 128, 6)),
              ("HEX_PRISM", (13, 17, 1)), ("HEX_PRISM", (9, 22, 3)), ("HEX_PRISM", (11, 10, 5))]


@pytest.mark.parametrize("shape,shpar", ALL_SHAPES)
def test_targets_bit_exact_against_oracle(D, shape, shpar):
    ctx = D.Context(-1)
    n, box = ctx.dda_setup_shape(shape, shpar)
    sites, origin = ctx.dda_get_sites()
    ref = o_tgt.make_target(shape, shpar)
    assert n == ref.n and box == ref.box
    np.testing.assert_array_equal(sites, ref.ijk)
    np.testing.assert_array_equal(origin, ref.origin)


def test_site_list_target_reorders_and_rejects_duplicates(D):
    ref = o_tgt.ellipsoid(5, 6, 7)
    rng = np.random.default_rng(5)
    perm = rng.permutation(ref.n)
    ctx = D.Context(-1)
    ctx.dda_setup_target(ref.ijk[perm] + np.array([3, -2, 7]), origin=(0.5, 0.5, 0.5))
    sites, origin = ctx.dda_get_sites()
    np.testing.assert_array_equal(sites, ref.ijk)
    np.testing.assert_allclose(origin, [3.5, -1.5, 7.5])
    dup = np.vstack([ref.ijk, ref.ijk[:1]])
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_setup_target(dup)
    assert ei.value.status == D.DDA_EINVAL


def test_site_list_targets_in_sequence_and_sorted_duplicates(D):
    """One context given several site lists in turn (its host buffers are reused between calls):
    each call's sites are exactly the new list's, in x-fastest order; a list in that order with a
    repeated site is rejected like an unordered one."""
    ctx = D.Context(-1)
    for s in [(5, 6, 7), (9, 4, 3), (5, 6, 7), (2, 2, 2)]:
        ref = o_tgt.ellipsoid(*s)
        ctx.dda_setup_target(ref.ijk, origin=(0.0, 0.0, 0.0))
        sites, _ = ctx.dda_get_sites()
        np.testing.assert_array_equal(sites, ref.ijk)
        assert ctx.n == ref.n
    ref = o_tgt.ellipsoid(5, 6, 7)
    dup = np.vstack([ref.ijk[:4], ref.ijk[3:4], ref.ijk[4:]])  # sorted, site 3 twice
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_setup_target(dup)
    assert ei.value.status == D.DDA_EINVAL


def test_invalid_arguments_and_state(D):
    ctx = D.Context(-1)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_set_incident(0.3, [(0, 0, 0)])
    assert ei.value.status == D.DDA_ESTATE
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_setup_shape("ELLIPSOID", (5.5, 6, 7))
    assert ei.value.status == D.DDA_EINVAL
    with pytest.raises(D.DDAError):
        ctx.dda_setup_shape("CYLINDER1", (5, 6, 4))
    ctx.dda_setup_shape("ELLIPSOID", (5, 6, 7))
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_set_incident(-1.0, [(0, 0, 0)])
    assert ei.value.status == D.DDA_EINVAL
    with pytest.raises(D.DDAError):  # e01 along the propagation direction
        ctx.dda_set_incident(0.3, [(0, 0, 0)], e01_lf=((1, 0), (0, 0), (0, 0)))
    ctx.dda_set_incident(0.3, [(0, 0, 0)])
    with pytest.raises(D.DDAError) as ei:  # host-only context has no device
        ctx.dda_build_green_fft()
    assert ei.value.status == D.DDA_ESTATE


def test_incidence_matches_oracle(D):
    ori = W.uniform_orientations(7, 99)
    for shape, shpar in [("RCTGLPRSM", (4, 5, 6)), ("HEX_PRISM", (6, 8, 4)), ("CYLINDER1", (5, 6, 3))]:
        ctx = D.Context(-1)
        ctx.dda_setup_shape(shape, shpar)
        for e01 in (((0, 0), (1, 0), (0, 0)), ((0, 0), (0.6, 0.1), (0.3, -0.7))):
            ctx.dda_set_incident(0.37, ori, e01, 2)
            k, e = ctx.dda_get_incidence()
            t = o_tgt.make_target(shape, shpar)
            e01c = np.array([complex(*c) for c in e01])
            for i, orr in enumerate(ori):
                k_ref, pols, _, _ = o_ori.incidence(0.37, orr, t.a1, t.a2, e01c, 2)
                np.testing.assert_allclose(k[2 * i], k_ref, atol=1e-15)
                np.testing.assert_allclose(k[2 * i + 1], k_ref, atol=1e-15)
                np.testing.assert_allclose(e[2 * i], pols[0], atol=1e-15)
                np.testing.assert_allclose(e[2 * i + 1], pols[1], atol=1e-15)


@pytest.mark.parametrize("presc", ["CM", "LATTDR", "GKDLDR"])
def test_polarizability_matches_oracle(D, presc):
    ori = W.uniform_orientations(5, 98)
    ctx = D.Context(-1)
    ctx.dda_setup_shape("ELLIPSOID", (6, 7, 8))
    ctx.dda_set_incident(0.41, ori, ((0, 0), (0.8, 0.0), (0.0, 0.6)), 2)
    ms = [1.33 + 0.01j, 2.5 + 1.5j, 0.9656 + 1.8628j]
    ctx.dda_set_polarizability(presc, ms)
    ia = ctx.dda_get_inv_alpha()
    k, e = ctx.dda_get_incidence()
    for b in range(ctx.nrhs):
        for c, m in enumerate(ms):
            ref = o_pol.inv_alpha(presc, m, 0.41, k[b] / 0.41, e[b])
            np.testing.assert_allclose(ia[b, c], ref, rtol=1e-14)


def test_orientation_grid_matches_oracle(D):
    """The library's orientation sampling against the oracle's restatement of the guide."""
    from oracle import orientation as oori
    for args in [((0, 90), 2, (0, 90), 3, (0, 180), 2), ((0, 360), 3, (0, 180), 5, (0, 360), 4),
                 ((10, 20), 1, (30, 150), 4, (0, 0), 1), ((0, 0), 1, (0, 0), 1, (0, 0), 1)]:
        ori, w = D.dda_orientation_grid(*args)
        ref, wr = oori.orientation_grid(*args)
        np.testing.assert_allclose(ori, np.array(ref), rtol=0, atol=1e-13)
        np.testing.assert_allclose(w, wr, rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape,shpar", [("ELLIPSOID", (12, 12, 12)), ("RCTGLPRSM", (32, 64, 64)),
                                         ("HEX_PRISM", (160, 128, 6))])
def test_kd_from_size_parameter_matches_oracle(D, shape, shpar):
    """kd = x / (a_eff / d), a_eff = (3 N / 4 pi)^(1/3) d, from the library; the oracle's a_eff is pinned
    to the guide's worked example (d / a_eff = 0.03173411 for the 32 x 64 x 64 block)."""
    ctx = D.Context(-1)
    ctx.dda_setup_shape(shape, shpar)
    ref = o_tgt.make_target(shape, shpar)
    for x in (1.0, 5.0, 20.0, 6.187):
        kd, aeff = ctx.dda_kd_from_x(x)
        assert aeff == pytest.approx(ref.aeff, rel=1e-15)
        assert kd == pytest.approx(x / ref.aeff, rel=1e-15)
    with pytest.raises(D.DDAError):
        ctx.dda_kd_from_x(0.0)
    with pytest.raises(D.DDAError):
        D.Context(-1).dda_kd_from_x(1.0)   # no target yet


def test_orientation_average_is_the_weighted_sum(D):
    """dda_orientation_average: <Q>_pol = sum_o w_o Q[o, pol], per polarization; written out as loops
    here; weights from the library's orientation grid and arbitrary ones."""
    ori, w = D.dda_orientation_grid((0, 360), 2, (0, 180), 3, (0, 360), 2)
    rng = np.random.default_rng(11)
    q = rng.standard_normal((len(w) * 2, 4))
    got = D.dda_orientation_average(q, w, 2)
    for pol in range(2):
        for k in range(4):
            ref = 0.0
            for o in range(len(w)):
                ref += w[o] * q[2 * o + pol, k]
            assert got[pol, k] == pytest.approx(ref, rel=1e-14, abs=1e-15)
    # constant per-orientation values average to themselves (the weights sum to one)
    const = np.tile(np.array([[1.5, -2.0, 0.25]]), (len(w) * 2, 1))
    np.testing.assert_allclose(D.dda_orientation_average(const, w, 2), np.array([[1.5, -2.0, 0.25]] * 2),
                               rtol=1e-14)
    # Mueller-shaped values, one polarization slot: [n_ori][ndir][16]
    m = rng.standard_normal((len(w), 3, 16))
    got = D.dda_orientation_average(m, w, 1)
    assert got.shape == (1, 3, 16)
    np.testing.assert_allclose(got[0], np.einsum("o,odk->dk", w, m), rtol=1e-13, atol=1e-15)
    with pytest.raises(D.DDAError):
        D.dda_orientation_average(q, w, 3)


def test_periodicity_arguments(D):
    ctx = D.Context(-1)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_set_periodicity(5.0, 0.0)    # no target yet
    assert ei.value.status == D.DDA_ESTATE
    ctx.dda_setup_shape("ELLIPSOID", (6, 5, 4))
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_set_periodicity(3.0, 0.0)    # shorter than the cell's y extent
    assert ei.value.status == D.DDA_EINVAL
    with pytest.raises(D.DDAError):
        ctx.dda_set_periodicity(8.0, 0.0, gamma=0.0)
    ctx.dda_set_periodicity(8.0, 0.0, 0.02)
    ctx.dda_set_periodicity(0.0, 0.0)        # finite again


def test_device_entry_points_refuse_a_host_only_context(D):
    """Every call that does device work, reached through the C ABI with a fully set-up host-only
    context, returns a status (DDA_ESTATE: no device, no Green tensor) before touching its buffer
    arguments; the context stays usable afterwards.  The buffers here are host memory on purpose:
    a call that went on to launch work would fault or fail with a CUDA error instead."""
    import ctypes
    L = D.LIB
    ctx = D.Context(-1)
    ctx.dda_setup_shape("ELLIPSOID", (5, 6, 7))
    kd, _ = ctx.dda_kd_from_x(1.0)
    ctx.dda_set_incident(kd, [(0, 0, 0), (0.3, 0.2, 0.1)])
    ctx.dda_set_polarizability("LATTDR", 1.5 + 0.1j)
    h, n, nrhs = ctx._h, ctx.n, ctx.nrhs
    alpha_before = ctx.dda_get_inv_alpha()
    buf = np.zeros(nrhs * 3 * n * 2 + 64)
    pb = buf.ctypes.data_as(ctypes.c_void_p)
    out = np.zeros(4096)
    po = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    i32 = np.zeros(64, dtype=np.int32)
    pi = i32.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    opts = D.dda_solve_opts(D.SOLVERS["BICGSTAB"], D.PRECISIONS["MIXED"], 1e-5, 100, 0.0, 0.0, 0, 8, 0, 1,
                            D.PRECONDS["NONE"], 0)
    reps = (D.dda_solve_report * nrhs)()
    handles = (ctypes.c_void_p * 1)(h.value)
    bufs = (ctypes.c_void_p * 1)(pb.value)
    sts = (ctypes.c_int * 1)(-1)
    calls = {
        "dda_incident_field": lambda: L.dda_incident_field(h, pb, D.DDA_C128),
        "dda_build_green_fft": lambda: L.dda_build_green_fft(h, None),
        "dda_matvec": lambda: L.dda_matvec(h, pb, pb, nrhs, D.DDA_C128),
        "dda_matvec (double-float)": lambda: L.dda_matvec(h, pb, pb, nrhs, D.DDA_C128DF),
        "dda_matvec_noalloc": lambda: L.dda_matvec_noalloc(h, pb, pb, nrhs, D.DDA_C64),
        "dda_solve": lambda: L.dda_solve(h, ctypes.byref(opts), pb, reps),
        "dda_solve_batch": lambda: L.dda_solve_batch(handles, 1, ctypes.byref(opts), bufs, None, sts),
        "dda_cross_sections": lambda: L.dda_cross_sections(h, pb, po, None, 0, None),
        "dda_profile_matvec": lambda: L.dda_profile_matvec(h, nrhs, D.DDA_C64, 1, po, pi),
        "dda_schedule_info": lambda: L.dda_schedule_info(h, D.DDA_C64, pi),
        "dda_angular_averages": lambda: L.dda_angular_averages(h, pb, ctypes.c_double(0.5), po, pi),
        "dda_force_torque": lambda: L.dda_force_torque(h, pb, ctypes.c_double(0.5), po, pi),
        "dda_near_field": lambda: L.dda_near_field(h, pb, po, ctypes.c_int64(1), po, None),
        "dda_periodic_scattering": lambda: L.dda_periodic_scattering(h, pb, 1, po, None, None, None),
    }
    for name, call in calls.items():
        assert call() == D.DDA_ESTATE, (name, L.dda_last_error(h))
        assert L.dda_last_error(h), name
    assert not np.any(buf), "a refused call wrote into its buffer"
    np.testing.assert_array_equal(ctx.dda_get_inv_alpha(), alpha_before)
    assert ctx.dda_kd_from_x(1.0)[0] == kd


def test_degenerate_inputs_on_the_host(D):
    """Empty and one-site targets, non-finite indices and beams: each is refused with DDA_EINVAL
    or, where it is a valid problem (one dipole, a one-cell shape), accepted with the right sizes."""
    ctx = D.Context(-1)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_setup_target(np.zeros((0, 3), dtype=np.int32))
    assert ei.value.status == D.DDA_EINVAL
    ctx.dda_setup_target(np.array([[3, -2, 7]], dtype=np.int32))
    n, box = ctx.dda_get_box()
    assert n == 1 and tuple(box) == (1, 1, 1)
    for shape in ("ELLIPSOID", "RCTGLPRSM", "CYLINDER1", "HEX_PRISM"):
        ctx.dda_setup_shape(shape, (1, 1, 1))
        assert ctx.n == 1, shape
    for bad in (float("nan"), float("inf"), 0.0, -1.0):
        with pytest.raises(D.DDAError) as ei:
            ctx.dda_set_incident(bad, [(0, 0, 0)])
        assert ei.value.status == D.DDA_EINVAL, bad
    ctx.dda_set_incident(0.3, [(0, 0, 0), (0.1, 0.2, 0.3)])
    for m in (complex(float("nan"), 0.0), complex(1.5, float("inf")), 1.0 + 0j):
        with pytest.raises(D.DDAError) as ei:
            ctx.dda_set_polarizability("LATTDR", m)
        assert ei.value.status == D.DDA_EINVAL, m
    # eps = m^2 = -2 is the pole of the Clausius-Mossotti alpha; 1/alpha stays finite there
    ctx.dda_set_polarizability("CM", 1j * math.sqrt(2.0))
    assert np.all(np.isfinite(ctx.dda_get_inv_alpha()))


def test_null_arguments_give_einval_with_a_message(D):
    """A NULL buffer or an out-of-range size is refused with DDA_EINVAL before anything else, and
    dda_last_error names the entry point (the header's convention for every non-const context)."""
    import ctypes
    L = D.LIB
    ctx = D.Context(-1)
    h = ctx._h
    out = np.zeros(64)
    po = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    calls = {
        "dda_incident_field": lambda: L.dda_incident_field(h, None, D.DDA_C128),
        "dda_get_inv_alpha": lambda: L.dda_get_inv_alpha(h, None),
        "dda_matvec": lambda: L.dda_matvec(h, None, None, 1, D.DDA_C64),
        "dda_matvec_noalloc": lambda: L.dda_matvec_noalloc(h, None, None, 1, D.DDA_C64),
        "dda_solve": lambda: L.dda_solve(h, None, None, None),
        "dda_cross_sections": lambda: L.dda_cross_sections(h, None, po, None, 0, None),
        "dda_profile_matvec": lambda: L.dda_profile_matvec(h, 1, D.DDA_C64, 0, po, None),
        "dda_schedule_info": lambda: L.dda_schedule_info(h, D.DDA_C64, None),
        "dda_angular_averages": lambda: L.dda_angular_averages(h, None, ctypes.c_double(0.5), po, None),
        "dda_force_torque": lambda: L.dda_force_torque(h, po, ctypes.c_double(-1.0), po, None),
        "dda_near_field": lambda: L.dda_near_field(h, po, po, ctypes.c_int64(0), po, None),
        "dda_periodic_scattering": lambda: L.dda_periodic_scattering(h, po, 0, po, None, None, None),
    }
    for name, call in calls.items():
        assert call() == D.DDA_EINVAL, name
        assert name.encode() in L.dda_last_error(h), (name, L.dda_last_error(h))
    # const-context getters report the status only
    assert L.dda_kd_from_x(h, ctypes.c_double(-1.0), None, None) == D.DDA_EINVAL

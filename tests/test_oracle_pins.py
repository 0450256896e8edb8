"""Pins for the FP64 oracle: values, closed forms and invariants fixed independently of it.

Each test names what fixes the expected value: a number printed in the DDSCAT
7.1 guide or in Bohren & Huffman, a textbook closed form written here in a
different form than the oracle uses, brute force on tiny inputs, or an exact
invariant of the mathematics.
"""
import math

import functools

import numpy as np
import pytest
import scipy.special as sp

from conftest import load_golden
from oracle import dda, interaction, mie, observables, orientation, polarizability, solvers, targets
from paper_1002_1505_gb300 import workloads as W


# ----------------------------------------------------------------------------- Mie

def test_mie_matches_bohren_huffman_printed_example():
    g, _ = load_golden("mie_bohren_huffman.txt")
    x = 2 * math.pi * g["radius"] / g["wavelength"]
    q = mie.efficiencies(complex(g["m_re"], g["m_im"]), x)
    assert q["Qext"] == pytest.approx(g["Qext"], abs=1e-5)
    assert q["Qsca"] == pytest.approx(g["Qsca"], abs=1e-5)
    assert q["Qback"] == pytest.approx(g["Qback"], abs=1e-5)


def test_mie_riccati_bessel_against_scipy():
    # upward recurrence is used only up to n_stop = x + 4 x^(1/3) + 2, where it is stable
    for x in (0.3, 2.0, 11.7):
        nstop = int(round(x + 4 * x ** (1 / 3) + 2))
        psi, chi = mie.riccati_bessel(x, nstop)
        n = np.arange(nstop + 1)
        np.testing.assert_allclose(psi, x * sp.spherical_jn(n, x), rtol=1e-7, atol=1e-10)
        np.testing.assert_allclose(chi, -x * sp.spherical_yn(n, x), rtol=1e-9)


def test_mie_rayleigh_limit():
    m = 1.5 + 0.2j
    x = 1e-3
    lor = (m * m - 1) / (m * m + 2)
    q = mie.efficiencies(m, x)
    assert q["Qabs"] == pytest.approx(4 * x * lor.imag, rel=1e-4)
    assert q["Qsca"] == pytest.approx(8.0 / 3.0 * x ** 4 * abs(lor) ** 2, rel=1e-4)


def test_mie_real_index_and_extinction_paradox():
    q = mie.efficiencies(1.33, 3.0)
    assert q["Qabs"] == pytest.approx(0.0, abs=1e-12)
    # opaque and large: Q_ext -> 2, the edge correction falling like x^(-2/3)
    d300 = mie.efficiencies(1.5 + 0.5j, 300.0)["Qext"] - 2.0
    d3000 = mie.efficiencies(1.5 + 0.5j, 3000.0)["Qext"] - 2.0
    assert 0 < d3000 < 0.02 and d300 / d3000 == pytest.approx(10 ** (2 / 3), rel=0.1)


# ----------------------------------------------------------------------------- targets

def _brute_count_ellipsoid(s):
    # plain loop over cell centres with exact rationals
    from fractions import Fraction as F
    n = 0
    for i in range(s[0]):
        for j in range(s[1]):
            for k in range(s[2]):
                x = F(2 * i + 1 - s[0], 2)
                y = F(2 * j + 1 - s[1], 2)
                z = F(2 * k + 1 - s[2], 2)
                if (x / s[0]) ** 2 + (y / s[1]) ** 2 + (z / s[2]) ** 2 <= F(1, 4):
                    n += 1
    return n


@pytest.mark.parametrize("s", [(12, 12, 12), (7, 5, 9), (6, 11, 4)])
def test_ellipsoid_count_brute_force(s):
    assert targets.ellipsoid(*s).n == _brute_count_ellipsoid(s)


def test_sphere12_has_912_sites_and_cubic_symmetry():
    t = targets.ellipsoid(12, 12, 12)
    assert t.n == 912 and t.box == (12, 12, 12)
    r = t.r
    key = set(map(tuple, np.round(r * 2).astype(int)))
    for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1)):
        assert set(map(tuple, np.round(r[:, perm] * 2).astype(int))) == key
    assert set(map(tuple, np.round(-r * 2).astype(int))) == key


def test_worked_example_target_bookkeeping():
    g, _ = load_golden("au_block_worked_example.txt")
    t = targets.rctglprsm(32, 64, 64)
    assert t.n == int(g["NAT0"])
    assert 1.0 / t.aeff == pytest.approx(g["d_over_aeff"], abs=2e-8)
    kd = g["k_aeff"] / t.aeff
    assert kd == pytest.approx(g["kd"], abs=1e-5)
    assert abs(0.9656 + 1.8628j) * kd == pytest.approx(g["mkd"], abs=1e-4)
    # TF origin at the centre of the upper x face: x spans [-32, 0]
    assert t.r[:, 0].min() == -31.5 and t.r[:, 0].max() == -0.5


def test_hex_prism_against_float_polygon():
    # point-in-hexagon by half-plane tests with floating-point vertices, skipping the
    # (absent) points within 1e-9 of an edge; independent of the integer formulation
    length, vv = 6, 14
    t = targets.hex_prism(length, vv, 6)  # a1 || z, a2 || y (face normal), a3 = -x (vertex)
    side = vv / 2.0
    verts = [(side * math.cos(math.pi / 3 * i), side * math.sin(math.pi / 3 * i)) for i in range(6)]
    # vertices along +-x (a3 axis), faces normal to y
    got = set(map(tuple, np.round(t.r * 2).astype(int)))
    exp = set()
    for i in range(vv):
        for j in range(vv):
            x = i + 0.5 - vv / 2
            y = j + 0.5 - vv / 2
            inside = True
            for a in range(6):
                (x0, y0), (x1, y1) = verts[a], verts[(a + 1) % 6]
                cross = (x1 - x0) * (y - y0) - (y1 - y0) * (x - x0)
                assert abs(cross) > 1e-9
                inside &= cross > 0
            if inside:
                for kk in range(length):
                    exp.add((int(round(2 * x)), int(round(2 * y)), 2 * kk + 1 - length))
    assert got == exp


def test_cylinder_count_brute_force():
    t = targets.cylinder1(5, 8, 2)  # axis along y
    n = 0
    for i in range(8):
        for k in range(8):
            x = i + 0.5 - 4
            z = k + 0.5 - 4
            n += (x * x + z * z <= 16.0)
    assert t.n == 5 * n and t.box[1] == 5


# ----------------------------------------------------------------------------- orientation

def test_orientation_examples_printed_in_guide():
    # Theta=90, Phi=0, beta=0: a1 = y_LF, a2 = -x_LF ; beta=90: a1 = y_LF, a2 = z_LF
    a1, a2, a3 = orientation.target_axes_in_lf(0.0, math.pi / 2, 0.0)
    np.testing.assert_allclose(a1, [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(a2, [-1, 0, 0], atol=1e-15)
    a1, a2, a3 = orientation.target_axes_in_lf(math.pi / 2, math.pi / 2, 0.0)
    np.testing.assert_allclose(a1, [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(a2, [0, 0, 1], atol=1e-15)
    # Phi = 90 puts a1 in the x_LF, z_LF plane
    a1, _, _ = orientation.target_axes_in_lf(0.3, 0.7, math.pi / 2)
    assert abs(a1[1]) < 1e-15


def test_orientation_inverse_relations_are_the_transpose():
    rng = np.random.default_rng(3)
    for _ in range(5):
        b, t, p = rng.uniform(0, 2 * math.pi, 3)
        a_lf = np.array(orientation.target_axes_in_lf(b, t, p))      # rows a_i in LF
        lab = np.array(orientation.lab_axes_in_tf(b, t, p, [1, 0, 0], [0, 1, 0]))  # x,y,z_LF in TF
        np.testing.assert_allclose(a_lf @ a_lf.T, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(lab, a_lf.T, atol=1e-14)
        assert np.linalg.det(a_lf) == pytest.approx(1.0)


def test_polarization_states_printed_in_guide():
    e1, e2 = orientation.polarizations_lf([0, 1, 0])
    np.testing.assert_allclose(e2, [0, 0, 1])
    e1, e2 = orientation.polarizations_lf([0, 1, 1j])  # (y + i z)/sqrt2 -> e02 = (i y + z)/sqrt2
    np.testing.assert_allclose(e1, np.array([0, 1, 1j]) / math.sqrt(2))
    np.testing.assert_allclose(e2, np.array([0, 1j, 1]) / math.sqrt(2))


# ----------------------------------------------------------------------------- polarizability

@pytest.mark.parametrize("presc", ["CM", "LATTDR", "GKDLDR"])
def test_alpha_real_index_is_lossless(presc):
    kd = 0.37
    ia = polarizability.inv_alpha(presc, 1.7, kd, [0.3, 0.4, math.sqrt(0.75)], [1, 0, 0])
    np.testing.assert_allclose(ia.imag, -2.0 / 3.0 * kd ** 3, rtol=1e-13)


@pytest.mark.parametrize("presc", ["LATTDR", "GKDLDR"])
def test_alpha_ldr_tends_to_clausius_mossotti(presc):
    m = 1.5 + 0.3j
    eps = m * m
    a_cm = 3 / (4 * math.pi) * (eps - 1) / (eps + 2)  # Lorentz-Lorenz, written out here
    ia = polarizability.inv_alpha(presc, m, 1e-6, [1, 0, 0], [0, 1, 0])
    np.testing.assert_allclose(1.0 / ia, a_cm, rtol=1e-10)


def test_gkdldr_equals_lattdr_for_axis_aligned_incidence_transverse_axes():
    # khat = x, e = y: LATTDR's S = 0, and GKDLDR's y and z entries use khat_y^2 = khat_z^2 = 0
    ia_l = polarizability.inv_alpha("LATTDR", 1.3 + 0.1j, 0.4, [1, 0, 0], [0, 1, 0])
    ia_g = polarizability.inv_alpha("GKDLDR", 1.3 + 0.1j, 0.4, [1, 0, 0], [0, 1, 0])
    np.testing.assert_allclose(ia_g[1:], ia_l[1:], rtol=1e-15)
    assert abs(ia_g[0] - ia_l[0]) > 1e-3


def _lattdr_s(ia, m, kd):
    """Recover Draine & Goodman's S from a LATTDR 1/alpha: the k^2 term is linear in S with slope
    eps b3 k^2 (b3 = -1.7700004, the coefficient printed in Draine & Goodman 1993, eq. 4.1)."""
    eps = m * m
    s0 = polarizability.inv_alpha("LATTDR", m, kd, [1, 0, 0], [0, 1, 0])[0]  # S = 0 exactly here
    return complex((ia - s0) / (eps * -1.7700004 * kd * kd))


def test_lattdr_s_term_hand_value_off_axis():
    # khat = (1,1,0)/sqrt2, e = (1,-1,0)/sqrt2: S = sum_a khat_a^2 e_a^2 = 1/4 + 1/4 = 1/2, while the
    # plausible misreading S = (khat . e)^2 gives 0.  The expected 1/alpha was worked out by hand from
    # Draine & Goodman (1993) eq. 4.1 with m = 1.5 + 0.1i, kd = 0.5, S = 1/2:
    #   1/alpha_CM = (4 pi / 3)(eps + 2)/(eps - 1),  + (b1 + eps b2 + eps b3 / 2) kd^2 - (2/3) i kd^3.
    r2 = math.sqrt(0.5)
    ia = polarizability.inv_alpha("LATTDR", 1.5 + 0.1j, 0.5, [r2, r2, 0], [r2, -r2, 0])
    np.testing.assert_allclose(ia, 12.886410816460371 - 2.4535841920447807j, rtol=1e-13)
    assert abs(_lattdr_s(ia[0], 1.5 + 0.1j, 0.5) - 0.5) < 1e-12


def test_lattdr_s_term_sums_to_one_minus_khat4_over_the_transverse_pair():
    # For any khat and two polarizations e1, e2 that with khat form an orthonormal (unitary) basis,
    # sum_pol |e_a|^2 = 1 - khat_a^2 for each axis a, so S(e1) + S(e2) = 1 - sum_a khat_a^4.
    # Holds for linear and for circular pairs; the squared-complex reading (e_a^2 without modulus)
    # fails it for circular ones, the (khat . e)^2 reading for every pair.
    rng = np.random.default_rng(7)
    m, kd = 1.33 + 0.05j, 0.3
    for _ in range(6):
        k = rng.standard_normal(3)
        k /= np.linalg.norm(k)
        u = np.cross(k, rng.standard_normal(3))
        u /= np.linalg.norm(u)
        v = np.cross(k, u)
        for e1 in (u.astype(complex), (u + 1j * v) / math.sqrt(2),
                   (math.cos(0.3) * u + 1j * math.sin(0.3) * v)):
            e2 = np.cross(np.conj(e1), k)          # orthogonal to e1 and k in the Hermitian sense
            assert abs(np.vdot(e1, e2)) < 1e-14 and abs(np.linalg.norm(e2) - 1) < 1e-14
            s1 = _lattdr_s(polarizability.inv_alpha("LATTDR", m, kd, k, e1)[0], m, kd)
            s2 = _lattdr_s(polarizability.inv_alpha("LATTDR", m, kd, k, e2)[0], m, kd)
            assert abs(s1 + s2 - (1 - np.sum(k ** 4))) < 1e-10
            assert abs(s1.imag) < 1e-12


def test_lattdr_s_term_circular_is_the_mean_of_the_linear_pair():
    # e = (y + i z)/sqrt2: S = (khat_y^2 + khat_z^2)/2, the mean of S(y) = khat_y^2 and S(z) = khat_z^2
    # (an intensity-weighted reading of the dispersion relation for an elliptical field).
    k = np.array([0.48, 0.6, 0.64])
    m, kd = 2.0 + 0.4j, 0.45
    s_circ = _lattdr_s(polarizability.inv_alpha("LATTDR", m, kd, k, np.array([0, 1, 1j]) / math.sqrt(2))[0], m, kd)
    assert abs(s_circ - (0.6 ** 2 + 0.64 ** 2) / 2) < 1e-12
    s_y = _lattdr_s(polarizability.inv_alpha("LATTDR", m, kd, k, [0, 1, 0])[0], m, kd)
    assert abs(s_y - 0.36) < 1e-12


# ----------------------------------------------------------------------------- interaction

def _dipole_field(rvec, p, k):
    """Field at rvec of a point dipole p at the origin (Jackson eq. 9.18, Gaussian units)."""
    r = np.linalg.norm(rvec)
    n = rvec / r
    return np.exp(1j * k * r) * (k * k * np.cross(np.cross(n, p), n) / r
                                 + (3 * n * np.dot(n, p) - p) * (1 / r ** 3 - 1j * k / r ** 2))


def test_two_dipole_blocks_are_minus_the_dipole_field():
    r = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, -1.5]])
    k = 0.8
    ia = np.array([[2.0 - 0.1j, 2.1 - 0.2j, 1.9 - 0.15j]] * 2)
    a = interaction.dense_matrix(r, k, ia).reshape(3, 2, 3, 2)
    for c in range(3):
        p = np.zeros(3, complex)
        p[c] = 1.0
        e = _dipole_field(r[0] - r[1], p, k)      # field at site 0 from unit dipole at site 1
        np.testing.assert_allclose(a[:, 0, c, 1], -e, rtol=1e-13)
        np.testing.assert_allclose(a[:, 0, c, 0], np.diag(ia[0])[:, c], rtol=0)


def test_single_dipole_cross_sections_closed_form():
    kd = 0.9
    m = 1.6 + 0.4j
    t = targets.from_sites([[0, 0, 0]], [0.0, 0.0, 0.0])
    prob = dda.build_problem(None, None, m, None, "CM", [(0, 0, 0)], target=t, kd=kd)
    ps, _ = dda.solve(prob, "lu")
    alpha = 1.0 / prob.rhs[0].inv_alpha[0, 0]
    aeff2 = t.aeff ** 2
    q = dda.cross_sections(prob, ps)[0]
    assert q["Qext"] * math.pi * aeff2 == pytest.approx(4 * math.pi * kd * alpha.imag, rel=1e-12)
    # scattered power of an oscillating dipole: C_sca = (8 pi / 3) k^4 |alpha|^2
    assert q["Qsca"] * math.pi * aeff2 == pytest.approx(8 * math.pi / 3 * kd ** 4 * abs(alpha) ** 2, rel=1e-12)
    c_int, g1, _, _, _ = observables.angular_averages(kd, t.r, ps[0], prob.rhs[0].axes, 1.0, 0.05)
    assert c_int == pytest.approx(8 * math.pi / 3 * kd ** 4 * abs(alpha) ** 2, rel=2e-3)
    assert abs(g1) < 2e-3  # dipole pattern is symmetric forward/backward


@pytest.mark.parametrize("shape,shpar,pad", [("ELLIPSOID", (5, 7, 9), None),
                                             ("ELLIPSOID", (5, 7, 9), (12, 15, 20)),
                                             ("CYLINDER1", (7, 6, 3), None)])
def test_fft_convolution_equals_direct_sum(shape, shpar, pad):
    prob = dda.build_problem(shape, shpar, 1.4 + 0.2j, 2.0, "GKDLDR", [(0.3, 1.1, 2.0)], pad=pad)
    p = W.seeded_vector((3, prob.target.n), 11)
    a = dda.apply_a(prob, 0, p, "direct")
    b = dda.apply_a(prob, 0, p, "fft")
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_matrix_is_complex_symmetric():
    prob = dda.build_problem("ELLIPSOID", (5, 6, 4), 1.4 + 0.2j, 2.0, "GKDLDR", [(0, 0, 0)])
    u = W.seeded_vector((3, prob.target.n), 1)
    v = W.seeded_vector((3, prob.target.n), 2)
    lhs = np.sum(u * dda.apply_a(prob, 0, v, "direct"))
    rhs = np.sum(v * dda.apply_a(prob, 0, u, "direct"))
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


# ----------------------------------------------------------------------------- solvers

def test_lu_bicgstab_ccg_agree_sphere12():
    w = W.SPHERE12
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    p_lu, _ = dda.solve(prob, "lu")
    p_bi, _ = dda.solve(prob, "bicgstab", tol=1e-12)
    p_cg, _ = dda.solve(prob, "ccg", tol=1e-12)
    for a, b, c in zip(p_lu, p_bi, p_cg):
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-9
        assert np.linalg.norm(a - c) / np.linalg.norm(a) < 1e-9
    # the returned P really solves A P = E: residual from an independent direct product
    r = prob.rhs[0].e_inc - dda.apply_a(prob, 0, p_bi[0], "direct")
    assert np.linalg.norm(r) / np.linalg.norm(prob.rhs[0].e_inc) < 1e-11


def test_bicgstab_l_reduces_to_bicgstab_and_solves():
    """BiCGstab(l) (Sleijpen & Fokkema 1993; the guide's PBCGS2 family): with l = 1 it is BiCGstab
    step for step (same iterates up to rounding), and with l = 2, 4 it converges to the LU solution."""
    w = W.SPHERE12
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    rh = prob.rhs[1]
    shape = rh.e_inc.shape

    def op(v):
        return dda.apply_a(prob, 1, v.reshape(shape), "direct").reshape(-1)
    e = rh.e_inc.reshape(-1)
    x1, it1, h1 = solvers.bicgstab_l(op, e, ell=1, tol=1e-10)
    xb, itb, hb = solvers.bicgstab(op, e, tol=1e-10)
    # bicgstab may stop on its half step; compare the residual histories where both are full steps
    n = min(len(h1), len(hb)) - 1
    assert n >= 5
    assert np.allclose(h1[:n], hb[:n], rtol=1e-6, atol=0)
    p_lu = solvers.lu_solve(interaction.dense_matrix(prob.target.r, prob.kd, rh.inv_alpha), e)
    for ell in (2, 4):
        x, it, h = solvers.bicgstab_l(op, e, ell=ell, tol=1e-12)
        assert h[-1] <= 1e-12 and it % ell == 0
        assert np.linalg.norm(x - p_lu) / np.linalg.norm(p_lu) < 1e-9
        # the recursive residual is the true one
        assert np.linalg.norm(e - op(x)) / np.linalg.norm(e) < 1e-11
    p2, its = dda.solve(prob, "bicgstab2", tol=1e-10)
    assert all(i > 0 for i in its)


def _sphere12_operator(index=0):
    w = W.SPHERE12
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    rh = prob.rhs[index]
    shape = rh.e_inc.shape

    def op(v):
        return dda.apply_a(prob, index, v.reshape(shape), "direct").reshape(-1)
    p_lu = solvers.lu_solve(interaction.dense_matrix(prob.target.r, prob.kd, rh.inv_alpha), rh.e_inc.reshape(-1))
    return op, rh.e_inc.reshape(-1), p_lu


def test_cocg_and_qmr_cs_solve_the_dda_system():
    """COCG (van der Vorst & Melissen 1990) and QMR for complex symmetric systems (Freund 1992) reach
    the LU solution of the (complex symmetric, non-Hermitian) DDA system; with a conjugated inner
    product in place of x^T y neither would."""
    op, e, p_lu = _sphere12_operator(1)
    for fn in (solvers.cocg, solvers.qmr_cs):
        out = fn(op, e, tol=1e-12)
        x, hist = out[0], out[2]
        assert hist[-1] <= 1e-12, fn.__name__
        assert np.linalg.norm(x - p_lu) / np.linalg.norm(p_lu) < 1e-9, fn.__name__
        assert np.linalg.norm(e - op(x)) / np.linalg.norm(e) < 1e-11
    p, its = dda.solve(dda.build_problem(W.SPHERE12.shape, W.SPHERE12.shpar, W.SPHERE12.m, W.SPHERE12.x,
                                         W.SPHERE12.prescription, W.SPHERE12.orientations), "qmr_cs", tol=1e-10)
    assert all(i > 0 for i in its)


@pytest.mark.parametrize("solver", ["cocg", "qmr_cs"])
def test_symmetric_krylov_terminates_at_the_number_of_distinct_eigenvalues(solver):
    """Exact-arithmetic property of both methods: on A = diag(lambda) with k distinct complex
    eigenvalues (complex symmetric, not Hermitian) the residual vanishes after k products."""
    rng = np.random.default_rng(3)
    lam = np.array([1 + 1j, 2 - 0.5j, 3 + 0.2j, 0.5 + 2j, -1.5 + 0.7j])
    for k in (2, 3, 5):
        dg = np.repeat(lam[:k], 13)
        b = rng.normal(size=dg.size) + 1j * rng.normal(size=dg.size)
        out = getattr(solvers, solver)(lambda v: dg * v, b, tol=1e-12, maxit=50)
        assert out[1] == k and out[2][-1] <= 1e-12, (solver, k, out[1])
        np.testing.assert_allclose(out[0], b / dg, rtol=1e-11)


def test_normal_eq_ratio_closed_forms():
    """The guide's stopping quantity |A^H A P - A^H E| / |A^H E| (section "Error Tolerance"): on a
    diagonal A = diag(a) it is sqrt(sum |a_i|^2 |a_i p_i - e_i|^2) / sqrt(sum |a_i|^2 |e_i|^2), written
    out element by element; P = 0 and P = 2 A^{-1} E give exactly 1, the solution gives 0."""
    a = np.array([2.0 + 1.0j, -0.5 + 0.25j, 1.5 - 2.0j])
    e = np.array([1.0 - 1.0j, 0.5j, 3.0 + 0.0j])
    p = np.array([0.25 + 0.5j, 1.0 - 1.0j, -0.5 + 0.5j])
    op = lambda v: a * v
    # hand form: A^H r = conj(a) r elementwise, with r = a p - e
    num = math.sqrt(sum(abs(ai) ** 2 * abs(ai * pi - ei) ** 2 for ai, pi, ei in zip(a, p, e)))
    den = math.sqrt(sum(abs(ai) ** 2 * abs(ei) ** 2 for ai, ei in zip(a, e)))
    assert abs(solvers.normal_eq_ratio(op, p, e) - num / den) < 1e-14
    assert abs(solvers.normal_eq_ratio(op, np.zeros(3, complex), e) - 1.0) < 1e-15
    assert abs(solvers.normal_eq_ratio(op, 2 * e / a, e) - 1.0) < 1e-14
    assert solvers.normal_eq_ratio(op, e / a, e) < 1e-15


def test_normal_eq_ratio_on_the_dda_system():
    """On the complex-symmetric DDA matrix, A^H = conj(A conj(.)) must be the conjugate transpose of
    the dense matrix: the ratio equals |A^H (A P - E)| / |A^H E| formed with the explicit dense A^H,
    vanishes at the LU solution and is 1 at P = 0."""
    w = W.SPHERE12
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    rh = prob.rhs[0]
    a = interaction.dense_matrix(prob.target.r, prob.kd, rh.inv_alpha)
    e = rh.e_inc.reshape(-1)
    op = lambda v: a @ v
    p_lu = solvers.lu_solve(a, e)
    assert solvers.normal_eq_ratio(op, p_lu, e) < 1e-12
    assert abs(solvers.normal_eq_ratio(op, np.zeros_like(e), e) - 1.0) < 1e-14
    p = p_lu + 1e-3 * W.seeded_vector(e.shape, 5)
    ah = a.conj().T
    ref = np.linalg.norm(ah @ (a @ p - e)) / np.linalg.norm(ah @ e)
    assert abs(solvers.normal_eq_ratio(op, p, e) / ref - 1.0) < 1e-12


def test_qmr_cs_quasi_residual_bounds_the_residual():
    """The quasi-residual |tau_{n+1}| never increases (a growing least-squares problem) and, with unit
    2-norm Lanczos vectors, |E - A x_n| <= sqrt(n+1) |tau_{n+1}|."""
    op, e, _ = _sphere12_operator(0)
    _, it, hist, q = solvers.qmr_cs(op, e, tol=1e-12)
    assert it >= 5
    assert all(q[i + 1] <= q[i] * (1 + 1e-12) for i in range(len(q) - 1))
    assert all(hist[i] <= np.sqrt(i + 1) * q[i] * (1 + 1e-9) for i in range(len(hist)))


def test_compositions_assemble_per_site_and_axis():
    """Per-site and per-axis compositions: equal indices reduce to the homogeneous problem, relabelling
    compositions (with the index list permuted alike) changes nothing, real indices absorb nothing,
    and a single anisotropic dipole gives C_ext = 4 pi k Im sum_a alpha_aa |e_a|^2 exactly."""
    t = targets.make_target("ELLIPSOID", (6, 5, 4))
    ori = [(0.3, 0.7, 1.1)]
    base = dda.build_problem(None, None, 1.5 + 0.1j, 2.0, "GKDLDR", ori, target=t)
    same = dda.build_problem(None, None, [1.5 + 0.1j, 1.5 + 0.1j], 2.0, "GKDLDR", ori, target=t,
                             comp=(t.ijk[:, 2] % 2))
    for a, b in zip(base.rhs, same.rhs):
        assert np.array_equal(a.inv_alpha, b.inv_alpha)
    c3 = np.stack([t.ijk[:, 2] % 2, np.zeros(t.n, int), (t.ijk[:, 0] + t.ijk[:, 1]) % 3], axis=1)
    m = [1.5 + 0.1j, 1.3 + 0.02j, 2.0 + 0.4j]
    p1 = dda.build_problem(None, None, m, 2.0, "LATTDR", ori, target=t, comp=c3)
    perm = np.array([2, 0, 1])                     # new label of old composition i
    m2 = [None] * 3
    for i, k in enumerate(perm):
        m2[k] = m[i]
    p2 = dda.build_problem(None, None, m2, 2.0, "LATTDR", ori, target=t, comp=perm[c3])
    for a, b in zip(p1.rhs, p2.rhs):
        assert np.array_equal(a.inv_alpha, b.inv_alpha)
    q1 = dda.cross_sections(p1, dda.solve(p1, "lu")[0])
    pr = dda.build_problem(None, None, [1.5, 1.3, 2.0], 2.0, "LATTDR", ori, target=t, comp=c3)
    for q in dda.cross_sections(pr, dda.solve(pr, "lu")[0]):
        assert abs(q["Qabs"]) < 1e-12 * q["Qext"]
    assert all(q["Qabs"] > 0 for q in q1)
    # one anisotropic site
    t1 = targets.from_sites([[0, 0, 0]], [0.0, 0.0, 0.0])
    kd = 0.3
    prob = dda.build_problem(None, None, m, None, "CM", [(0.2, 0.9, 0.4)], target=t1, kd=kd, comp=[[0, 1, 2]])
    ps, _ = dda.solve(prob, "lu")
    for rh, q in zip(prob.rhs, dda.cross_sections(prob, ps)):
        alpha = 1.0 / rh.inv_alpha[0]
        cext = 4 * math.pi * kd * np.sum(alpha.imag * np.abs(rh.e_tf) ** 2)
        assert q["Qext"] * math.pi * t1.aeff ** 2 == pytest.approx(cext, rel=1e-12)


def test_orientation_grid_guide_examples():
    """The guide's own examples of the (beta, Theta, Phi) sampling, and the weights' quadrature."""
    deg = lambda v: [math.degrees(x) for x in v]
    oris, _ = orientation.orientation_grid((0, 90), 2, (0, 0), 1, (0, 0), 1)
    assert deg([o[0] for o in oris]) == pytest.approx([22.5, 67.5])
    oris, _ = orientation.orientation_grid((0, 0), 1, (0, 0), 1, (0, 180), 2)
    assert deg([o[2] for o in oris]) == pytest.approx([45.0, 135.0])
    oris, _ = orientation.orientation_grid((0, 0), 1, (0, 90), 3, (0, 0), 1)
    assert deg([o[1] for o in oris]) == pytest.approx([0.0, 60.0, 90.0], abs=1e-12)
    oris, _ = orientation.orientation_grid((0, 0), 1, (0, 90), 2, (0, 0), 1)
    assert deg([o[1] for o in oris]) == pytest.approx([41.4096, 75.5225], abs=1e-4)
    # weights sum to one; odd NTHETA integrates cubics in cos(Theta) exactly over [-1, 1]
    oris, w = orientation.orientation_grid((0, 360), 3, (0, 180), 5, (0, 360), 4)
    assert len(oris) == 60 and w.sum() == pytest.approx(1.0, abs=1e-15)
    ct = np.cos([o[1] for o in oris])
    for k, exact in ((1, 0.0), (2, 1.0 / 3.0), (3, 0.0)):
        assert np.sum(w * ct ** k) == pytest.approx(exact, abs=1e-14)
    # even NTHETA: midpoint rule, exact for linear functions
    oris, w = orientation.orientation_grid((0, 360), 1, (0, 180), 4, (0, 360), 1)
    assert np.sum(w * np.cos([o[1] for o in oris])) == pytest.approx(0.0, abs=1e-15)


# ----------------------------------------------------------------------------- observables

def test_real_index_has_zero_absorption():
    prob = dda.build_problem("ELLIPSOID", (6, 6, 6), 1.5, 2.0, "LATTDR", [(0.2, 0.4, 0.9)])
    ps, _ = dda.solve(prob, "lu")
    for q in dda.cross_sections(prob, ps):
        assert abs(q["Qabs"]) < 1e-13 * q["Qext"]


def test_optical_theorem_against_angular_integration():
    prob = dda.build_problem("ELLIPSOID", (8, 6, 5), 1.5 + 0.1j, 2.0, "GKDLDR", [(0.2, 0.4, 0.9)])
    ps, _ = dda.solve(prob, "lu")
    q = dda.cross_sections(prob, ps)
    geo = math.pi * prob.target.aeff ** 2
    for i in range(2):
        c_int, _, _, _, _ = observables.angular_averages(prob.kd, prob.target.r, ps[i], prob.rhs[i].axes,
                                                         prob.x, 0.1)
        assert c_int / geo == pytest.approx(q[i]["Qsca"], rel=2e-3)


def test_efficiencies_invariant_under_phase_origin():
    w = W.SPHERE12
    t0 = targets.ellipsoid(6, 7, 5)
    t1 = targets.Target(ijk=t0.ijk, box=t0.box, origin=t0.origin + np.array([0.3, -1.7, 2.2]),
                        a1=t0.a1, a2=t0.a2)
    out = []
    for t in (t0, t1):
        prob = dda.build_problem(None, None, 1.4 + 0.3j, None, "GKDLDR", [(0.4, 0.8, 1.9)], target=t, kd=0.5)
        ps, _ = dda.solve(prob, "lu")
        out.append(dda.cross_sections(prob, ps))
    for a, b in zip(*out):
        for key in a:
            assert a[key] == pytest.approx(b[key], rel=1e-11, abs=1e-14)


def test_sphere_cubic_rotation_gives_same_efficiencies():
    w = W.SPHERE12
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription,
                             [(0, 0, 0), (0, math.pi / 2, 0), (math.pi / 2, math.pi / 2, math.pi / 2)])
    ps, _ = dda.solve(prob, "bicgstab", tol=1e-12)
    q = dda.cross_sections(prob, ps)
    for qi in q[1:]:
        assert qi["Qext"] == pytest.approx(q[0]["Qext"], rel=1e-9)
        assert qi["Qabs"] == pytest.approx(q[0]["Qabs"], rel=1e-9)


def test_dda_converges_to_mie_as_dipole_count_grows():
    m, x = 1.33 + 0.01j, 1.0
    exact = mie.efficiencies(m, x)
    errs = []
    for d in (8, 12, 16, 24):
        prob = dda.build_problem("ELLIPSOID", (d, d, d), m, x, "LATTDR", [(0, 0, 0)], iorth=1)
        ps, _ = dda.solve(prob, "bicgstab", tol=1e-10)
        q = dda.cross_sections(prob, ps)[0]
        errs.append(abs(q["Qext"] / exact["Qext"] - 1))
    assert errs[-1] < 0.01                 # "within a few percent" for |m|kd << 1
    assert errs[0] > errs[-1]
    assert all(e2 < e1 * 1.05 for e1, e2 in zip(errs, errs[1:]))


def test_dda_small_sphere_rayleigh_scaling():
    m = 1.5 + 0.1j
    lor = (m * m - 1) / (m * m + 2)
    qs = []
    for x in (0.02, 0.04):
        prob = dda.build_problem("ELLIPSOID", (10, 10, 10), m, x, "LATTDR", [(0, 0, 0)], iorth=1)
        ps, _ = dda.solve(prob, "lu")
        qs.append(dda.cross_sections(prob, ps)[0])
    # Q_sca / x^4 and Q_abs / x are size-independent in the Rayleigh limit
    assert qs[0]["Qsca"] / 0.02 ** 4 == pytest.approx(qs[1]["Qsca"] / 0.04 ** 4, rel=2e-3)
    assert qs[0]["Qabs"] / 0.02 == pytest.approx(qs[1]["Qabs"] / 0.04, rel=2e-3)
    # and close to the continuum sphere's values (pseudosphere shape error of a few %)
    assert qs[0]["Qabs"] == pytest.approx(4 * 0.02 * lor.imag, rel=0.05)
    assert qs[0]["Qsca"] == pytest.approx(8 / 3 * 0.02 ** 4 * abs(lor) ** 2, rel=0.05)


def test_quadrature_direction_count_matches_worked_example():
    g, _ = load_golden("au_block_worked_example.txt")
    rings = observables.scattering_angles(g["k_aeff"], 0.5)
    assert sum(len(ph) for _, ph, _ in rings) == int(g["NAVG"])
    total = sum(w * len(ph) for _, ph, w in rings)
    assert total == pytest.approx(4 * math.pi, rel=1e-14)


def test_mueller_relations_for_a_single_dipole():
    # one isotropic dipole: S_11(theta) = k^2 dC/dOmega = k^6 |alpha|^2 (1 + cos^2)/2 for
    # unpolarized light; S_12 = -(sin^2)/2 ... ; written from the textbook dipole pattern
    kd = 0.7
    t = targets.from_sites([[0, 0, 0]], [0.0, 0.0, 0.0])
    prob = dda.build_problem(None, None, 1.3 + 0.2j, None, "CM", [(0, 0, 0)], target=t, kd=kd)
    ps, _ = dda.solve(prob, "lu")
    alpha = 1.0 / prob.rhs[0].inv_alpha[0, 0]
    for th in (0.0, 0.5, 1.3, 2.9):
        mm = dda.mueller(prob, ps, [(th, 0.4)])[0]
        i0 = kd ** 6 * abs(alpha) ** 2
        assert mm[0, 0] == pytest.approx(i0 * (1 + math.cos(th) ** 2) / 2, rel=1e-12)
        assert mm[0, 1] == pytest.approx(-i0 * math.sin(th) ** 2 / 2, rel=1e-10, abs=1e-14 * i0)
        assert mm[2, 2] == pytest.approx(i0 * math.cos(th), rel=1e-10, abs=1e-14 * i0)


@pytest.mark.slow
def test_worked_example_au_block():
    """The guide's sample calculation (RCTGLPRSM 32x64x64 Au block, GKDLDR)."""
    g, rows = load_golden("au_block_worked_example.txt")
    w = W.AU_BLOCK
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    ps, _ = dda.solve(prob, "bicgstab", tol=1e-6, workers=-1)
    qs = dda.cross_sections(prob, ps)
    ka = prob.kd * prob.target.aeff
    for q in qs:  # the two polarizations are equivalent for this block
        assert q["Qext"] == pytest.approx(g["Qext"], rel=1e-4)
        assert q["Qabs"] == pytest.approx(g["Qabs"], rel=1e-4)
        assert q["Qsca"] == pytest.approx(g["Qsca"], rel=1e-4)
        assert q["Qpha"] == pytest.approx(g["Qpha"], rel=2e-4)
    dirs = [(math.radians(r[0]), math.radians(r[1])) for r in rows]
    mm = dda.mueller(prob, ps, dirs)
    for r, m in zip(rows, mm):
        assert m[0, 0] == pytest.approx(r[2], rel=5e-4)
        assert m[0, 1] == pytest.approx(r[3], rel=5e-4, abs=5e-3)
        assert m[1, 0] == pytest.approx(m[0, 1], rel=1e-9, abs=1e-9)
        assert m[1, 1] == pytest.approx(r[5], rel=5e-4)
    back = [m for r, m in zip(rows, mm) if r[0] == 180][0]
    assert back[0, 0] / (math.pi * ka ** 2) == pytest.approx(g["Qbk"], rel=1e-4)


# ----------------------------------------------------------------------------- force and torque

def test_imaginary_part_of_the_dipole_field_is_a_plane_wave_integral():
    """Im G(R) = (k^3 / 4 pi) oint (I - n n) exp(i k n.R) dOmega (the identity behind the far-field
    torque), against the closed-form tensor, including R -> 0 where it is (2/3) k^3 I."""
    from oracle import forces
    k = 0.7
    dirs, w = forces.gauss_directions(40, 80)
    for R in ([1.0, 0.0, 0.0], [0.3, -1.2, 2.0], [3.5, 2.5, -0.5]):
        R = np.array(R)
        quad = sum(wi * (np.eye(3) - np.outer(n, n)) * np.exp(1j * k * n @ R) for n, wi in zip(dirs, w))
        quad *= k ** 3 / (4 * np.pi)
        np.testing.assert_allclose(quad.real, np.imag(forces.field_tensor(R[None, :], k)[0]), atol=1e-12)
        assert np.abs(quad.imag).max() < 1e-12
    quad0 = k ** 3 / (4 * np.pi) * sum(wi * (np.eye(3) - np.outer(n, n)) for n, wi in zip(dirs, w))
    np.testing.assert_allclose(quad0, 2.0 / 3.0 * k ** 3 * np.eye(3), atol=1e-13)


def test_far_field_force_and_torque_equal_the_site_by_site_sums():
    """Arbitrary dipole moments on a small irregular array: force and torque from the incident field,
    the full dipole-dipole field with its gradient and the radiation reaction, site by site, equal
    the incident part plus the far-field integrals (a dropped term, a sign or a transposed T fails)."""
    from oracle import forces
    rng = np.random.default_rng(4)
    r = rng.integers(-3, 4, size=(14, 3)).astype(float)
    r = np.unique(r, axis=0) + np.array([0.5, 0.0, -0.5])
    n = r.shape[0]
    k = 0.6
    khat = np.array([0.36, 0.48, 0.8])
    e = np.cross(khat, [0.0, 0.0, 1.0]) + 0.4j * np.cross(khat, np.cross(khat, [0.0, 0.0, 1.0]))
    e /= np.linalg.norm(e)
    e_inc = e[:, None] * np.exp(1j * k * (r @ khat))[None, :]
    p = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    Fd, Gd = forces.direct_force_torque(k, r, p, e_inc, k * khat)
    dirs, w = forces.gauss_directions(40, 80)
    Ff, Gf = forces.far_field_force_torque(k, r, p, e_inc, k * khat, dirs, w)
    np.testing.assert_allclose(Ff, Fd, rtol=0, atol=2e-8 * np.abs(Fd).max())
    np.testing.assert_allclose(Gf, Gd, rtol=0, atol=2e-8 * np.abs(Gd).max())


def test_single_dipole_circular_torque_is_the_absorbed_angular_momentum():
    """One dipole, circularly polarized wave along z: each absorbed photon brings hbar, so
    Q_Gamma = Q_abs khat exactly (and the transverse force and torque vanish)."""
    from oracle import forces
    k = 0.45
    alpha = 0.08 + 0.015j
    e = np.array([1.0, 1j, 0.0]) / math.sqrt(2)
    khat = np.array([0.0, 0.0, 1.0])
    p = (alpha * e)[:, None]
    e_inc = e[:, None]
    r = np.zeros((1, 3))
    dirs, w = forces.gauss_directions(24, 48)
    F, G = forces.far_field_force_torque(k, r, p, e_inc, k * khat, dirs, w)
    aeff = (3 / (4 * np.pi)) ** (1 / 3)
    qpr, qg = forces.efficiency_vectors(k, aeff, F, G)
    c_ext = 4 * np.pi * k * alpha.imag
    c_sca = 8 * np.pi / 3 * k ** 4 * abs(alpha) ** 2
    q_abs = (c_ext - c_sca) / (np.pi * aeff ** 2)
    np.testing.assert_allclose(qg, [0, 0, q_abs], atol=1e-12 * abs(q_abs) + 1e-15)
    np.testing.assert_allclose(qpr, [0, 0, c_ext / (np.pi * aeff ** 2)], atol=1e-12)  # dipole pattern: g = 0


def test_torque_on_a_solved_sphere_vanishes_for_linear_and_not_for_circular_light():
    """A DDA pseudosphere (cubic symmetry, incidence along a lattice axis): with linear polarization
    mirror symmetry forbids any torque; with circular polarization the torque is along khat and,
    the sphere being nearly isotropic and small, close to Q_abs (photons absorbed)."""
    from oracle import forces
    for e01, circ in (([0, 0], [1, 0], [0, 0]), False), (([0, 0], [1, 0], [0, 1]), True):
        prob = dda.build_problem("ELLIPSOID", (6, 6, 6), 1.5 + 0.3j, 0.8, "LATTDR", [(0, 0, 0)], e01_lf=e01, iorth=1)
        ps, _ = dda.solve(prob, "lu")
        rh = prob.rhs[0]
        dirs, w = forces.gauss_directions(32, 64)
        F, G = forces.far_field_force_torque(prob.kd, prob.target.r, ps[0], rh.e_inc, rh.k_tf, dirs, w)
        qpr, qg = forces.efficiency_vectors(prob.kd, prob.target.aeff, F, G)
        q = dda.cross_sections(prob, ps)[0]
        khat = rh.k_tf / np.linalg.norm(rh.k_tf)
        assert 0 < np.dot(qpr, khat) <= q["Qext"] + 1e-12  # Q_ext - Q_sca <cos>, with <cos> >= 0 here
        assert np.linalg.norm(qpr - np.dot(qpr, khat) * khat) < 1e-8 * q["Qext"]
        if not circ:
            assert np.linalg.norm(qg) < 1e-9 * q["Qabs"]
        else:
            assert np.linalg.norm(qg - np.dot(qg, khat) * khat) < 1e-8 * q["Qabs"]
            assert abs(np.dot(qg, khat)) == pytest.approx(q["Qabs"], rel=0.02)


# ----------------------------------------------------------------------------- rotated dielectric frames

def _aniso_target():
    t = targets.make_target("ELLIPSOID", (6, 5, 4))
    comp = np.stack([t.ijk[:, 0] % 2, (t.ijk[:, 1] + 1) % 3, np.full(t.n, 2)], axis=1)
    return t, comp


@pytest.mark.parametrize("presc", ["CM", "LATTDR", "GKDLDR"])
def test_dielectric_frame_reduces_to_aligned_materials(presc):
    """Zero angles: the ANIFRMFIL tensor is the TF-aligned per-axis composition exactly; angles
    (pi/2, 0, 0) put e_1 on y_TF and e_2 on -x_TF, i.e. the aligned case with the compositions of x and
    y swapped."""
    t, comp = _aniso_target()
    m = [1.5 + 0.1j, 1.33 + 0.01j, 2.2 + 0.6j]
    ori = W.uniform_orientations(1, 81)
    ref = dda.build_problem(None, None, m, 2.0, presc, ori, target=t, comp=comp)
    rot0 = dda.build_problem(None, None, m, 2.0, presc, ori, target=t, comp=comp, df_angles=np.zeros((t.n, 3)))
    sw = dda.build_problem(None, None, m, 2.0, presc, ori, target=t, comp=comp[:, [1, 0, 2]],
                           df_angles=np.tile([math.pi / 2, 0.0, 0.0], (t.n, 1)))
    for b in range(2):
        diag = np.stack([np.diag(ref.rhs[b].inv_alpha[j]) for j in range(t.n)]) if ref.rhs[b].inv_alpha.ndim == 3 \
            else ref.rhs[b].inv_alpha
        for prob in (rot0, sw):
            ia = prob.rhs[b].inv_alpha
            assert ia.shape == (t.n, 3, 3)
            np.testing.assert_allclose(np.einsum("jaa->ja", ia), diag, rtol=1e-14, atol=1e-14)
            off = ia - np.einsum("ja,ab->jab", np.einsum("jaa->ja", ia), np.eye(3))
            assert np.abs(off).max() < 1e-13


def test_rotated_dielectric_tensor_is_symmetric_and_lossless_for_real_indices():
    t, comp = _aniso_target()
    rng = np.random.default_rng(8)
    ang = rng.uniform(0, 2 * math.pi, size=(t.n, 3))
    prob = dda.build_problem(None, None, [1.5, 1.33, 2.2], 2.0, "LATTDR", W.uniform_orientations(1, 82), target=t,
                             comp=comp, df_angles=ang)
    ia = prob.rhs[0].inv_alpha
    np.testing.assert_allclose(ia, np.transpose(ia, (0, 2, 1)), atol=1e-14)
    # sum_a e_a e_a^T = I and Im d_a = -(2/3) k^3 for real m: Im(alpha^{-1}) = -(2/3) k^3 I
    np.testing.assert_allclose(ia.imag, np.broadcast_to(-2 / 3 * prob.kd ** 3 * np.eye(3), ia.shape), atol=1e-14)
    ps, _ = dda.solve(prob, "lu")
    assert abs(dda.cross_sections(prob, ps)[0]["Qabs"]) < 1e-12


def test_single_rotated_uniaxial_dipole_extinction_closed_form():
    """One site of a uniaxial material (c-axis 30 degrees from x_TF in the x-z plane, like the guide's
    ANIFRMFIL example): alpha = sum_a (1/d_a) e_a e_a^T, so C_ext = 4 pi k sum_a Im(1/d_a) |e_a . E|^2."""
    from oracle import forces  # noqa: F401  (module import check only)
    t = targets.Target(ijk=np.zeros((1, 3), dtype=np.int64), box=(1, 1, 1), origin=np.zeros(3),
                       a1=np.array([1.0, 0, 0]), a2=np.array([0, 1.0, 0]))
    m = [1.7 + 0.2j, 1.4 + 0.05j]
    ang = np.array([[0.5236, math.pi / 2, 0.0]])
    comp = np.array([[0, 1, 1]])
    kd = 0.3
    prob = dda.build_problem(None, None, m, None, "CM", [(0.4, 1.1, 0.2)], target=t, kd=kd, comp=comp, df_angles=ang)
    for rh in prob.rhs:
        ps, _ = dda.solve(dda.Problem(target=t, kd=kd, x=prob.x, rhs=[rh], pad=prob.pad), "lu")
        q = observables.efficiencies(kd, t.aeff, rh.e_inc, ps[0], rh.inv_alpha)
        ct, st = math.cos(0.5236), math.sin(0.5236)
        e1 = np.array([ct, 0.0, st])          # phi_DF = 90 deg: e_1 in the x-z plane
        e2 = np.array([-st, 0.0, ct])
        e3 = np.array([0.0, -1.0, 0.0])
        c_ext = 0.0
        for e_a, mm in ((e1, m[0]), (e2, m[1]), (e3, m[1])):
            eps = mm * mm
            d = (4 * math.pi / 3) * (eps + 2) / (eps - 1) - 2j / 3 * kd ** 3  # CM with radiative reaction
            c_ext += 4 * math.pi * kd * (1 / d).imag * abs(np.dot(e_a, rh.e_inc[:, 0])) ** 2
        assert q["Qext"] == pytest.approx(c_ext / (math.pi * t.aeff ** 2), rel=1e-10)


# ----------------------------------------------------------------------------- near field (DDfield)

def test_dipole_fields_against_jackson_and_faraday():
    """The near-field formulas: E of one dipole equals the Jackson form used above for A_jk, and
    curl E = i k B (Faraday's law for exp(-i w t), Gaussian units) by central differences."""
    from oracle import nearfield
    k = 0.8
    p = np.array([0.3 + 0.2j, -1.0 + 0.1j, 0.5 - 0.4j])
    for x in ([1.3, -0.7, 2.1], [-3.0, 0.5, 0.25]):
        x = np.array(x)
        E, B = nearfield.dipole_fields(x[None, :], p[None, :], k)
        np.testing.assert_allclose(E[0], _dipole_field(x, p, k), rtol=1e-13)
        h = 1e-4
        def dEd(b):
            e = np.zeros(3)
            e[b] = h
            return (nearfield.dipole_fields((x + e)[None, :], p[None, :], k)[0][0] -
                    nearfield.dipole_fields((x - e)[None, :], p[None, :], k)[0][0]) / (2 * h)
        d0, d1, d2 = dEd(0), dEd(1), dEd(2)
        curl = np.array([d1[2] - d2[1], d2[0] - d0[2], d0[1] - d1[0]])
        np.testing.assert_allclose(curl, 1j * k * B[0], rtol=1e-6, atol=1e-9)


def test_near_field_far_limit_is_the_scattering_amplitude():
    """At a large distance R along n the dipole sum tends to exp(ikR)/R k^2 sum_j (P_j - n(n.P_j))
    exp(-ik n.r_j), the far field the efficiencies and Mueller matrix are built from."""
    from oracle import nearfield
    prob = dda.build_problem("ELLIPSOID", (5, 4, 6), 1.5 + 0.2j, 1.5, "LATTDR", [(0.3, 0.8, 1.1)], iorth=1)
    ps, _ = dda.solve(prob, "lu")
    rh = prob.rhs[0]
    n = np.array([0.36, -0.48, 0.8])
    R = 4.0e5
    E, _ = nearfield.fields_at([R * n], prob.kd, prob.target.r, ps[0], rh.k_tf, 0 * rh.e_tf)
    g = ps[0] @ np.exp(-1j * prob.kd * (prob.target.r @ n))
    far = np.exp(1j * prob.kd * R) / R * prob.kd ** 2 * (g - n * np.dot(n, g))
    np.testing.assert_allclose(E[0], far, rtol=2e-4, atol=1e-12 * np.abs(far).max())


@pytest.mark.slow
def test_near_field_of_the_au_block_matches_the_printed_track():
    """The guide's DDfield sample output (tests/golden/au_block_ddfield_track.txt) from the oracle's
    BiCGstab solution of the Au block: E_y within 2e-3 of the printed values (the guide's run was
    single precision at TOL 1e-5), E_x and E_z zero by symmetry."""
    from oracle import nearfield
    _, rows = load_golden("au_block_ddfield_track.txt")
    w = W.AU_BLOCK
    prob = dda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations, iorth=1)
    ps, _ = dda.solve(prob, "bicgstab", tol=1e-7, workers=-1)
    rh = prob.rhs[0]
    pts = np.array([row[:3] for row in rows])
    E, _ = nearfield.fields_at(pts, prob.kd, prob.target.r, ps[0], rh.k_tf, rh.e_tf)
    for row, e in zip(rows, E):
        ref = complex(row[3], row[4])
        assert abs(e[1] - ref) <= 2e-3 * max(abs(ref), 0.1), (row, e[1])
        assert abs(e[0]) < 1e-6 and abs(e[2]) < 1e-6


# ----------------------------------------------------------------------------- periodic targets

def _tuc():
    return targets.make_target("ELLIPSOID", (3, 4, 3))


@pytest.mark.parametrize("periods", [(5.0, 6.0), (5.0, 0.0), (0.0, 7.0)])
def test_periodic_fft_product_equals_the_replica_sum(periods):
    """The FFT embedding of the periodic interaction A^per (every offset of the wrapped grid, Bloch
    phases, cutoff) against the plain O(N^2 x replicas) sum, at oblique incidence."""
    from oracle import periodic
    t = _tuc()
    prob = dda.build_problem(None, None, 1.5 + 0.2j, 1.0, "LATTDR", [(0.3, 1.0, 0.4)], target=t, periods=periods,
                             gamma=0.15)
    p = W.seeded_vector((3, t.n), 12)
    a1 = dda.apply_a(prob, 0, p, "direct")
    a2 = dda.apply_a(prob, 0, p, "fft")
    assert np.linalg.norm(a1 - a2) / np.linalg.norm(a1) < 1e-13
    # and it differs from the finite target's product (the replicas matter)
    fin = dda.build_problem(None, None, 1.5 + 0.2j, 1.0, "LATTDR", [(0.3, 1.0, 0.4)], target=t)
    assert np.linalg.norm(a1 - dda.apply_a(fin, 0, p, "direct")) / np.linalg.norm(a1) > 1e-3


def test_periodic_interaction_reciprocity():
    """A^per(r; k) = A^per(-r; -k) (the replicas' Bloch phases flip with the incidence), so
    u^T A(k) v = v^T A(-k) u; at normal incidence A^per is complex symmetric."""
    from oracle import periodic
    t = _tuc()
    k = np.array([0.2, 0.35, -0.15])
    u = W.seeded_vector((3, t.n), 3)
    v = W.seeded_vector((3, t.n), 4)
    ia = np.full((t.n, 3), 2.0 + 0.1j)
    av = periodic.matvec_direct(t.r, np.linalg.norm(k), ia, v, k, (5.0, 6.0), 0.15)
    au = periodic.matvec_direct(t.r, np.linalg.norm(k), ia, u, -k, (5.0, 6.0), 0.15)
    assert abs(np.sum(u * av) - np.sum(v * au)) < 1e-12 * abs(np.sum(u * av))


def test_periodic_slab_absorbs_like_a_fresnel_film():
    """An infinite slab (2-D periodic TUC of one column of 8 dipoles, periods 1 x 1) at normal
    incidence absorbs per unit area what the continuum film of the same index and thickness absorbs
    (Airy-Fresnel), within the DDA's discretization error (1 %); Draine & Flatau 2008 validate the
    periodic method the same way."""
    from oracle import periodic
    nl, m, kd = 8, 1.5 + 0.1j, 0.1
    tt = targets.Target(ijk=np.stack([np.arange(nl), np.zeros(nl, int), np.zeros(nl, int)], 1), box=(nl, 1, 1),
                        origin=np.zeros(3), a1=np.array([1.0, 0, 0]), a2=np.array([0, 1.0, 0]))
    pr = dda.build_problem(None, None, m, None, "LATTDR", [(0, 0, 0)], target=tt, kd=kd, iorth=1, periods=(1, 1),
                           gamma=0.08)
    ps, _ = dda.solve(pr, "lu")
    q = dda.cross_sections(pr, ps)[0]
    absorbed = q["Qabs"] * np.pi * tt.aeff ** 2 / (1.0 * 1.0)   # C_abs per unit-cell area
    assert absorbed == pytest.approx(periodic.slab_fresnel_absorption(m, kd, nl), rel=0.01)
    # every layer of the column carries the same field pattern as its replicas: P is uniform in y, z
    assert np.abs(ps[0][0]).max() < 1e-10 * np.abs(ps[0][1]).max()


# ----------------------------------------------------------------------------- periodic targets: orders

def _slab(nl=8):
    return targets.Target(ijk=np.stack([np.arange(nl), np.zeros(nl, int), np.zeros(nl, int)], 1), box=(nl, 1, 1),
                          origin=np.zeros(3), a1=np.array([1.0, 0, 0]), a2=np.array([0, 1.0, 0]))


@functools.lru_cache(maxsize=None)
def _solved_slab(m, kd=0.2, gamma=0.04):
    """The 8-layer slab (periods 1 x 1, normal incidence, LATTDR), solved by LU."""
    tt = _slab(8)
    pr = dda.build_problem(None, None, m, None, "LATTDR", [(0, 0, 0)], target=tt, kd=kd, iorth=2, periods=(1, 1),
                           gamma=gamma)
    ps, _ = dda.solve(pr, "lu")
    return tt, pr, ps


@pytest.mark.parametrize("m", [1.5 + 0.1j, 1.5 + 0.0j])
def test_periodic_slab_reflects_and_transmits_like_a_fresnel_film(m):
    """The slab of the absorption pin (one column of 8 dipoles, periods 1 x 1, normal incidence):
    the (0, 0) order's transmission and reflection coefficients against the Airy-Fresnel film of the
    same index and thickness (within the DDA's discretization error: measured 0.3 % at kd = 0.2), and
    T + R + A = 1, which holds for the DDA equations themselves as the interaction cutoff gamma -> 0
    (1.1e-5 at gamma = 0.04, 7e-7 at 0.02)."""
    from oracle import periodic
    nl, kd = 8, 0.2
    tt, pr, ps = _solved_slab(m)
    q = dda.cross_sections(pr, ps)
    rf, tf = periodic.slab_fresnel_rt(m, kd, nl)
    for i in range(2):
        t, r = periodic.transmission_reflection(pr, i, ps[i], 0, 0)
        a = q[i]["Qabs"] * np.pi * tt.aeff ** 2
        assert t == pytest.approx(tf, rel=5e-3)
        assert r == pytest.approx(rf, rel=5e-3)
        assert t + r + a == pytest.approx(1.0, abs=3e-5)
        # only the specular orders exist for periods of one lattice spacing at kd = 0.2
        assert periodic.transmission_reflection(pr, i, ps[i], 1, 0) is None


@pytest.mark.parametrize("ori,periods", [((0.0, 0.0, 0.0), (8, 8)), ((0.3, 0.5, 0.7), (8, 7))])
def test_periodic_orders_carry_the_incident_power(ori, periods):
    """A doubly periodic array of small ellipsoids whose periods admit several diffraction orders
    (kd = 1, periods 8 x 8 or 8 x 7, normal and oblique incidence): transmitted and reflected powers
    over every allowed order plus the absorbed power add up to the incident power (gamma = 0.005),
    and S^(2d)_11 times the flux ratio |n_x| / |n0_x| is the mean of the two polarizations' power in
    each order other than the (0, 0) transmission (which interferes with the incident wave)."""
    from oracle import periodic
    t = _tuc()
    pr = dda.build_problem(None, None, 1.4 + 0.05j, None, "GKDLDR", [ori], target=t, kd=1.0, iorth=2,
                           periods=periods, gamma=0.005)
    ps, _ = dda.solve(pr, "lu")
    q = dda.cross_sections(pr, ps)
    area = periods[0] * periods[1]
    k0 = pr.rhs[0].k_tf
    n0x = abs(k0[0]) / pr.kd
    allowed = [(M, N) for M in range(-3, 4) for N in range(-3, 4)
               if periodic.order_direction(k0, periods, M, N) is not None]
    assert len(allowed) >= 4 and (0, 0) in allowed
    for i in range(2):
        tot = q[i]["Qabs"] * np.pi * t.aeff ** 2 / (area * n0x)
        for M, N in allowed:
            tot += sum(periodic.transmission_reflection(pr, i, ps[i], M, N))
        assert tot == pytest.approx(1.0, abs=1e-6)
    for M, N in allowed:
        for sign in (1, -1):
            if (M, N) == (0, 0) and sign == 1:
                continue
            n = periodic.order_direction(k0, periods, M, N, sign=sign)
            s = periodic.mueller_in_order(pr, 0, ps, n)
            mean = np.mean([periodic.transmission_reflection(pr, i, ps[i], M, N)[0 if sign == 1 else 1]
                            for i in range(2)])
            assert s[0, 0] * abs(n[0]) / n0x == pytest.approx(mean, rel=1e-10)
    # the guide's condition on (M, N): |k_parallel + 2 pi (M, N) / L| < k exactly for the allowed orders
    for M in range(-3, 4):
        for N in range(-3, 4):
            kp = np.hypot(k0[1] + 2 * np.pi * M / periods[0], k0[2] + 2 * np.pi * N / periods[1])
            assert ((M, N) in allowed) == (kp < pr.kd)


@pytest.mark.parametrize("periods", [(8, 0), (0, 7)])
def test_periodic_cones_carry_the_scattered_power(periods):
    """A target periodic along one axis (small ellipsoids, period 8 along y or 7 along z, kd = 1,
    oblique incidence): the power per unit length leaving through a distant cylinder, integrated over
    the azimuth zeta of every allowed cone M from S^(1d) (I_sca = S^(1d) I_in / (k rho), radial flux
    fraction k_perp / k), equals the scattering cross section per unit length C_sca / L of the solved
    unit cell (unpolarized incidence), at gamma = 0.000625 (the one-dimensional lattice sums converge
    slowly in gamma)."""
    from oracle import periodic
    t = _tuc()
    pr = dda.build_problem(None, None, 1.4 + 0.05j, None, "GKDLDR", [(0.2, 0.6, 0.3)], target=t, kd=1.0, iorth=2,
                           periods=periods, gamma=0.000625)
    ps, _ = dda.solve(pr, "lu")
    q = dda.cross_sections(pr, ps)
    length = periods[0] or periods[1]
    axis = 1 if periods[0] else 2
    csca = np.mean([(q[i]["Qext"] - q[i]["Qabs"]) * np.pi * t.aeff ** 2 for i in range(2)]) / length
    nz = 240
    tot = 0.0
    cones = [M for M in range(-3, 4) if periodic.order_direction(pr.rhs[0].k_tf, periods, M) is not None]
    assert len(cones) >= 2
    for M in cones:
        for zeta in np.arange(nz) * 2 * np.pi / nz:
            n = periodic.order_direction(pr.rhs[0].k_tf, periods, M, zeta=zeta)
            assert abs(np.linalg.norm(n) - 1.0) < 1e-14
            s = periodic.mueller_in_order(pr, 0, ps, n)
            tot += s[0, 0] * np.sqrt(1.0 - n[axis] ** 2) / pr.kd * (2 * np.pi / nz)
    assert tot == pytest.approx(csca, rel=1e-4)


def test_periodic_near_field_away_from_the_slab_is_its_plane_waves():
    """The guide's DDfield for an infinite target: summing the replicas' dipole fields (cutoff
    exp[-(gamma k D)^4] on each) at points a wavelength or so in front of and behind the slab gives the
    plane waves of its (0, 0) orders -- incident plus reflected in front, transmitted behind -- whose
    amplitudes come from the independent Fourier-space sum (periodic.order_fields); E and B within
    2e-3 at gamma = 0.04 (the real-space sum converges as gamma -> 0: 3e-3 -> 2e-4 from 0.04 to 0.02
    at kd = 0.4)."""
    from oracle import nearfield, periodic
    tt, pr, ps = _solved_slab(1.5 + 0.1j)
    kd = pr.kd
    rh = pr.rhs[0]
    (nt, et), (nr, er) = periodic.order_fields(pr, 0, ps[0], 0, 0)
    pts = np.array([[-15.0, 0.3, 0.2], [25.0, 0.1, 0.7]])
    E, B = nearfield.fields_at(pts, kd, tt.r, ps[0], rh.k_tf, rh.e_tf, periods=(1, 1), gamma=0.04)
    x0 = pts[0]
    inc = rh.e_tf * np.exp(1j * np.dot(rh.k_tf, x0))
    refl = er * np.exp(1j * kd * np.dot(nr, x0))
    k0h = rh.k_tf / kd
    e_front, b_front = inc + refl, np.cross(k0h, inc) + np.cross(nr, refl)
    trans = et * np.exp(1j * kd * np.dot(nt, pts[1]))
    for got, ref in ((E[0], e_front), (B[0], b_front), (E[1], trans), (B[1], np.cross(nt, trans))):
        assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref)
    # and the reflected wave is really there: without it the front field is off by |r| ~ 0.3
    assert np.linalg.norm(E[0] - inc) > 0.2 * np.linalg.norm(inc)

"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a closed
form, a symmetry, a library routine, brute force on a tiny lattice, or the
convergence order of the integrator.  A plausible mistake in the oracle (a
dropped leaf, a wrong twist factor or sign, a transposed operand, a wrong RK
coefficient) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I
from tests import fields as F

TW = I.default_twist(1)
NOTW = np.zeros((4, 4), dtype=np.int64)
TINY = (2, 2, 6, 6)


def test_twist_eater_is_a_zero_action_stationary_point():
    """Sec. 1 twist relation: Gamma_1 Gamma_2 = Z_12 Gamma_2 Gamma_1, so Z* P = 1 on every plaquette."""
    g1, g2 = I.twist_matrices(1)
    w = np.exp(2j * math.pi / 3)
    assert np.allclose(g1 @ g2, w * g2 @ g1, atol=1e-15)
    for L in [(2, 2, 6, 6), (4, 4, 12, 12), (3, 3, 3, 3)]:
        U = I.twist_eater(L)
        m = O.measure(U, TW)
        assert abs(m["S"]) < 1e-12 and abs(m["E"]) < 1e-14 and abs(m["Q"]) < 1e-14
        assert abs(m["P"] - 1) < 1e-15
        assert np.abs(O.force(U, TW)).max() < 1e-14
        # with the twist switched off the same field has non-zero action: the factor matters
        assert O.measure(U, NOTW)["S"] > 1.0
        # the wrong centre element (k = -1) is not an eater either
        assert O.measure(U, I.default_twist(-1))["S"] > 1.0


def test_action_ordered_pairs_equals_twice_reduced():
    """S_W sums Tr[1 - Z* P] over ordered mu != nu (Sec. 3.1); its value is real and equals 2 s."""
    U = I.random_links(TINY, 11, 0.5)
    a = O.wilson_action_ordered(U, TW)
    assert abs(a.imag) < 1e-9
    assert a.real == pytest.approx(2 * O.reduced_action(U, TW), rel=1e-13)


def test_force_is_minus_twice_the_lie_derivative_of_s():
    """Z^a = -g0^2 d^a S_W = -2 d^a s by central differences on a 2x2x6x6 twisted lattice."""
    U = I.random_links(TINY, 1, 0.5)
    Z = O.force(U, TW)
    T = I.gell_mann() * 0.5j  # anti-Hermitian, tr(T^a T^b) = -delta/2
    h = 1e-5
    links = [(0, 0, 0, 0, 0), (0, 0, 0, 0, 1), (1, 2, 1, 0, 0), (2, 1, 0, 1, 1), (3, 4, 1, 1, 2),
             (5, 5, 0, 0, 3), (0, 0, 1, 0, 1), (0, 0, 0, 1, 0), (4, 3, 1, 1, 0), (1, 1, 1, 1, 1)]
    for (x3, x2, x1, x0, mu) in links:
        for a in range(8):
            def s_of(e):
                V = U.copy()
                V[x3, x2, x1, x0, mu] = scipy.linalg.expm(e * T[a]) @ U[x3, x2, x1, x0, mu]
                return O.reduced_action(V, TW)

            d = (s_of(h) - s_of(-h)) / (2 * h)
            za = -2 * np.trace(T[a] @ Z[x3, x2, x1, x0, mu]).real
            assert za == pytest.approx(-2 * d, abs=2e-6)


def test_force_is_traceless_antihermitian():
    Z = O.force(I.random_links(TINY, 4, 0.5), TW)
    assert np.abs(Z + O.dag(Z)).max() < 1e-14
    assert np.abs(O.tr(Z)).max() < 1e-14


def test_expm_matches_library_and_group_properties():
    rng = np.random.default_rng(0)
    for scale in [1e-3, 0.1, 1.0, 7.0]:
        A = rng.normal(size=(50, 3, 3)) + 1j * rng.normal(size=(50, 3, 3))
        X = scale * O.proj_ta(A)
        E = O.expm(X)
        ref = np.stack([scipy.linalg.expm(x) for x in X])
        assert np.abs(E - ref).max() < 1e-13 * max(1.0, math.exp(3 * scale))
        assert np.abs(E @ O.dag(E) - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(E) - 1).max() < 1e-13
        assert np.abs(E @ O.expm(-X) - np.eye(3)).max() < 1e-13
    G = rng.normal(size=(20, 3, 3)) + 1j * rng.normal(size=(20, 3, 3))
    ref = np.stack([scipy.linalg.expm(g) for g in G])
    assert np.abs(O.expm(G) - ref).max() < 1e-11 * np.abs(ref).max()


def test_flow_preserves_su3():
    U = I.random_links(TINY, 5, 0.6)
    for _ in range(5):
        U = O.rk3_step(U, 0.02, TW)
    assert np.abs(U @ O.dag(U) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_action_decreases_with_rate_minus_force_norm():
    """Gradient flow: ds/dt = -sum ||Z||_F^2 (central difference of s along the flow) and s monotone."""
    U = I.random_links(TINY, 2, 0.5)
    Z = O.force(U, TW)
    rate = -float(np.sum(np.abs(Z) ** 2))
    e = 1e-4
    sp = O.reduced_action(O.rk3_step(U, e, TW), TW)
    sm = O.reduced_action(O.rk3_step(U, -e, TW), TW)
    assert (sp - sm) / (2 * e) == pytest.approx(rate, rel=1e-6)
    s_prev = O.reduced_action(U, TW)
    for _ in range(10):
        U = O.rk3_step(U, 0.02, TW)
        s = O.reduced_action(U, TW)
        assert s < s_prev
        s_prev = s


def test_rk3_is_third_order():
    """Global error of E(t) shrinks by ~8 when eps halves (Luscher's RK3 is third order)."""
    U0 = I.random_links(TINY, 2, 0.5)
    T = 0.16

    def run(eps):
        U = U0.copy()
        for _ in range(int(round(T / eps))):
            U = O.rk3_step(U, eps, TW)
        return O.measure(U, TW)["E"], U

    eref, uref = run(0.00125)
    errs = [abs(run(eps)[0] - eref) for eps in (0.04, 0.02, 0.01)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 10.5 and 6.5 < r2 < 10.5, (r1, r2)


def test_gauge_invariance_along_the_flow():
    """Periodic gauge transforms commute with the twist factors: E, Q, P, S unchanged along the flow."""
    L = TINY
    U = I.random_links(L, 7, 0.5)
    Ug = F.gauge_transform(U, F.random_gauge(L, 99))
    for _ in range(3):
        a, b = O.measure(U, TW), O.measure(Ug, TW)
        for k in "EQPS":
            assert b[k] == pytest.approx(a[k], rel=1e-12, abs=1e-13)
        U, Ug = O.rk3_step(U, 0.05, TW), O.rk3_step(Ug, 0.05, TW)


def test_twisted_corner_can_be_moved_by_a_centre_change_of_variables():
    """Multiplying U_0 on the column x0 = 0, x1 = 1 by Z moves the twisted plaquettes to x1 = 1."""
    U = I.random_links(TINY, 8, 0.5)
    w = np.exp(2j * math.pi / 3)
    Up = U.copy()
    Up[:, :, 1, 0, 0] *= w
    a, b = O.measure(U, TW), O.measure(Up, TW, corner=(0, 1, 0, 0))
    for k in "EQPS":
        assert b[k] == pytest.approx(a[k], rel=1e-12, abs=1e-13)
    Ua = O.rk3_step(U, 0.05, TW)
    Ub = O.rk3_step(Up, 0.05, TW, corner=(0, 1, 0, 0))
    Ub[:, :, 1, 0, 0] *= np.conj(w)
    assert np.abs(Ua - Ub).max() < 1e-13


def test_reflection_flips_q_and_keeps_e():
    U = I.random_links((3, 3, 4, 5), 3, 0.4)
    a, b = O.measure(U, TW), O.measure(F.reflect_x3(U), TW)
    assert b["E"] == pytest.approx(a["E"], rel=1e-13)
    assert b["P"] == pytest.approx(a["P"], rel=1e-13)
    assert b["Q"] == pytest.approx(-a["Q"], rel=1e-10)
    assert abs(a["Q"]) > 1e-3


def test_complex_conjugation_with_opposite_twist():
    U = I.random_links(TINY, 6, 0.5)
    a, b = O.measure(U, TW), O.measure(np.conj(U), -TW)
    for k in "EQPS":
        assert b[k] == pytest.approx(a[k], rel=1e-12, abs=1e-13)


def test_single_link_clover_closed_form():
    """One link exp(i th lambda_3/2) on a periodic 3^4 lattice: 12 clover sites carry
    G = (+-1/4) diag(sin(th/2), -sin(th/2), 0), so sum_n E(n) = 3/2 sin^2(th/2); Q = 0;
    six plaquettes carry the link, s = 12 (1 - cos(th/2))."""
    L = (3, 3, 3, 3)
    V = 81
    for th in [0.3, 1.1]:
        for mu in range(4):
            m = O.measure(F.single_link(L, th, site=(1, 2, 0, 1), mu=mu), NOTW)
            assert m["E"] == pytest.approx(1.5 * math.sin(th / 2) ** 2 / V, rel=1e-13)
            assert abs(m["Q"]) < 1e-15
            assert m["S"] == pytest.approx(12 * (1 - math.cos(th / 2)), rel=1e-12)
            assert m["P"] == pytest.approx(1 - 12 * (1 - math.cos(th / 2)) / (18 * V), rel=1e-14)


@pytest.mark.parametrize("planes,sign", [(((0, 1), (2, 3)), +1), (((0, 2), (1, 3)), -1), (((0, 3), (1, 2)), +1)])
def test_constant_abelian_fields_fix_every_term_of_q(planes, sign):
    """Constant flux f_ab, f_cd in two complementary planes: G_ab = sin(f_ab H) at every site, so
    E = 2 sin^2 f_ab + 2 sin^2 f_cd and Q = eps_{abcd} V sin(f_ab) sin(f_cd) / (2 pi^2)  (eq. qlatt)."""
    L = (4, 4, 4, 4)
    V = 256
    U = F.unit_field(L)
    (a, b), (c, d) = planes
    U, f1 = F.abelian_flux(U, a, b, 1)
    U, f2 = F.abelian_flux(U, c, d, 2)
    m = O.measure(U, NOTW)
    assert m["E"] == pytest.approx(2 * math.sin(f1) ** 2 + 2 * math.sin(f2) ** 2, rel=1e-13)
    assert m["Q"] == pytest.approx(sign * V * math.sin(f1) * math.sin(f2) / (2 * math.pi ** 2), rel=1e-12)
    assert O.levi_civita(a, b, c, d) == sign


def test_traceless_clover_variant_differs_only_by_the_trace():
    U = I.random_links(TINY, 9, 0.5)
    G = O.field_strength(U, TW)
    Gt = O.field_strength(U, TW, traceless=True)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                d = G[mu][nu] - Gt[mu][nu]
                assert np.abs(d - d[..., 0:1, 0:1] * np.eye(3)).max() < 1e-14
                assert np.abs(O.tr(Gt[mu][nu])).max() < 1e-14
                assert np.abs(G[mu][nu] - O.dag(G[mu][nu])).max() < 1e-14


def test_flow_records_and_partial_final_step():
    U = I.random_links(TINY, 10, 0.3)
    n, rest = O.flow_steps(0.045, 0.01)
    assert n == 4 and rest == pytest.approx(0.005)
    Uf, rec = O.flow(U, 0.01, 0.045, TW)
    assert [r[0] for r in rec] == pytest.approx([0, 0.01, 0.02, 0.03, 0.04, 0.045])
    U2 = U
    for h in [0.01] * 4 + [rest]:
        U2 = O.rk3_step(U2, h, TW)
    assert np.abs(Uf - U2).max() == 0.0
    Ef = [r[1] for r in rec]
    assert all(x > y for x, y in zip(Ef, Ef[1:]))


# ---- time-slice charge q(x0, t) and its correlator (Sec. 4, eq. qcorr) ----------------------------

def test_slices_sum_to_q_and_parity_reverses_them():
    U = I.random_links((3, 3, 4, 5), 3, 0.4)
    q = O.slice_charge(U, TW, 3)
    assert q.shape == (5,)
    assert np.sum(q) == pytest.approx(O.measure(U, TW)["Q"], rel=1e-12, abs=1e-14)
    qr = O.slice_charge(F.reflect_x3(U), TW, 3)
    # x3 -> -x3 maps slice x to slice -x and flips the sign of the density
    assert np.allclose(qr, -q[(-np.arange(5)) % 5], rtol=1e-11, atol=1e-14)
    q2 = O.slice_charge(U, TW, 2)
    assert q2.shape == (4,) and np.sum(q2) == pytest.approx(np.sum(q), rel=1e-12, abs=1e-14)


def test_constant_abelian_field_has_uniform_slices():
    L = (4, 4, 4, 4)
    U = F.unit_field(L)
    U, f1 = F.abelian_flux(U, 0, 1, 1)
    U, f2 = F.abelian_flux(U, 2, 3, 2)
    q = O.slice_charge(U, NOTW, 3)
    Q = O.measure(U, NOTW)["Q"]
    assert np.allclose(q, Q / 4, rtol=1e-12)


def test_slice_correlator_symmetry_and_sum_rule():
    rng = np.random.default_rng(1)
    qs = rng.normal(size=(5, 12)) * 0.05
    Q = qs.sum(axis=1)
    C, kept = O.slice_correlator(qs, Q)
    assert kept == int(np.sum(np.abs(Q) < 0.5))
    # C(d) = C(T - d) and sum_d C(d) = <Q^2>/T over the kept configurations
    assert np.allclose(C[1:], C[1:][::-1], rtol=1e-13)
    keep = np.abs(Q) < 0.5
    assert np.sum(C) == pytest.approx(np.mean(Q[keep] ** 2) / 12, rel=1e-12)
    # brute-force double loop for one configuration
    one, _ = O.slice_correlator(qs[:1], [0.0])
    for d in range(12):
        ref = sum(qs[0][(x + d) % 12] * qs[0][x] for x in range(12)) / 12
        assert one[d] == pytest.approx(ref, rel=1e-13)
    assert O.slice_correlator(qs, [1.0] * 5) == (None, 0)

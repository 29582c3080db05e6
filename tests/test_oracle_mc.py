"""Pins of the Monte Carlo oracle (oracle/tgf_mc_oracle.py) against what mathematics fixes.

* the counter-based generator reproduces SplitMix64's published output;
* the quaternion form of SU(2) is a homomorphism and the SU(2) projection is the one that
  Re Tr[R M] sees (Re Tr[R M] = 2 (R x)_0 for every R in SU(2));
* the X0 sampler (Kennedy-Pendleton and Creutz branches) follows the density
  sqrt(1 - x^2) exp(alpha x): mean = I_2(alpha)/I_1(alpha) and a Kolmogorov-Smirnov test
  against the exact distribution function;
* the Cabibbo-Marinari heat-bath of one SU(3) link with staple s*1 reproduces <Re Tr U> of
  the one-link SU(3) integral (a sum of Toeplitz determinants of Bessel functions);
* over-relaxation keeps the twisted action exactly;
* at very large beta the heat-bath keeps the twist-eater (the classical minimum) within the
  thermal fluctuations that equipartition allows.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import iv

from oracle import tgf_mc_oracle as M
from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I


def test_counter_generator_is_splitmix64():
    ref = [int(x, 16) for x in open(__file__.replace("test_oracle_mc.py", "golden/splitmix64_seed0.txt")).read().split()
           if x.startswith("0x")]
    assert [int(v) for v in M.hash64(0, np.arange(len(ref)))] == ref
    u = M.uniform(12345, np.arange(100000))
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)


def _rand_quat(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def test_quaternions_are_su2_and_projection_matches_trace():
    rng = np.random.default_rng(1)
    a, b = _rand_quat(rng, 50), _rand_quat(rng, 50)
    A, B = M.q_to_mat(a), M.q_to_mat(b)
    np.testing.assert_allclose(M.q_to_mat(M.qmul(a, b)), A @ B, atol=1e-14)
    np.testing.assert_allclose(A @ np.conj(np.swapaxes(A, -1, -2)), np.broadcast_to(np.eye(2), A.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(A), 1.0, atol=1e-14)
    np.testing.assert_allclose(M.su2_part(A), a, atol=1e-15)
    Mx = rng.normal(size=(50, 2, 2)) + 1j * rng.normal(size=(50, 2, 2))
    x = M.su2_part(Mx)
    lhs = np.trace(A @ Mx, axis1=-2, axis2=-1).real
    np.testing.assert_allclose(lhs, 2 * M.qmul(a, x)[:, 0], atol=1e-13)


def _cdf(alpha):
    xs = np.linspace(-1, 1, 4001)
    w = np.sqrt(np.clip(1 - xs * xs, 0, None)) * np.exp(alpha * (xs - 1))
    c = integrate.cumulative_trapezoid(w, xs, initial=0.0)
    c /= c[-1]
    return lambda v: np.interp(v, xs, c)


@pytest.mark.parametrize("alpha", [0.3, 1.5, 3.0, 12.0, 60.0])
def test_x0_sampler_density(alpha):
    n = 40000
    c0 = np.arange(n, dtype=np.uint64) * np.uint64(M.SLOTS)
    x0, acc = M.sample_x0(np.full(n, alpha), 777, c0)
    assert acc.all()
    assert np.all(np.abs(x0) <= 1.0)
    mean = float(iv(2, alpha) / iv(1, alpha))
    assert abs(x0.mean() - mean) < 5 * x0.std() / math.sqrt(n)
    assert stats.kstest(x0, _cdf(alpha)).pvalue > 1e-3
    X = M.random_su2(x0, 777, c0)
    np.testing.assert_allclose(np.sum(X * X, axis=-1), 1.0, atol=1e-14)
    v = X[:, 1:]
    assert np.all(np.abs(v.mean(axis=0)) < 5 * math.sqrt((1 - (x0 ** 2).mean()) / 3 / n) + 1e-12)


@pytest.mark.parametrize("beta,s", [(3.0, 1.0), (6.0, 2.0)])
def test_one_link_heatbath_matches_su3_integral(beta, s):
    n, it, burn = 3000, 40, 10
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    S = s * np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    sites = np.arange(n)
    means = []
    for w in range(it):
        U = M._update_links(U, S, beta, "hb", M.config_key(5, 0), w, 0, n, sites)
        if w >= burn:
            means.append(np.trace(U, axis1=-2, axis2=-1).real)
    per_link = np.mean(means, axis=0)
    expect = M.su3_one_link_re_tr(beta * s / 3.0)
    assert abs(per_link.mean() - expect) < 5 * per_link.std() / math.sqrt(n)


def _lattice():
    L = (2, 2, 4, 4)
    U = I.random_links(L, 3, 0.8)
    return L, U, I.default_twist(1)


def test_overrelaxation_keeps_the_action():
    L, U, tw = _lattice()
    s0 = O.reduced_action(U, tw)
    V = M.sweep(U, tw, 5.0, "or")
    assert np.max(np.abs(V - U)) > 1e-2
    assert abs(O.reduced_action(V, tw) - s0) < 1e-11 * abs(s0)
    np.testing.assert_allclose(np.linalg.det(V), 1.0, atol=1e-13)


def test_heatbath_keeps_su3_and_changes_the_field():
    L, U, tw = _lattice()
    V = M.sweep(U, tw, 5.0, "hb", seed=9, cfg=2, sweep_index=4)
    assert np.max(np.abs(V - U)) > 1e-2
    np.testing.assert_allclose(np.linalg.det(V), 1.0, atol=1e-13)
    np.testing.assert_allclose(V @ np.conj(np.swapaxes(V, -1, -2)),
                               np.broadcast_to(np.eye(3), V.shape), atol=1e-13)
    # the same draws give the same field; another sweep number gives another one
    np.testing.assert_array_equal(V, M.sweep(U, tw, 5.0, "hb", seed=9, cfg=2, sweep_index=4))
    assert np.max(np.abs(V - M.sweep(U, tw, 5.0, "hb", seed=9, cfg=2, sweep_index=5))) > 1e-2


def test_heatbath_at_large_beta_stays_at_the_twist_eater():
    L = (2, 2, 4, 4)
    U = I.twist_eater(L, 1)
    tw = I.default_twist(1)
    assert abs(O.reduced_action(U, tw)) < 1e-12
    V = M.hybrid(U, tw, 1e7, 2, seed=1, cfg=0, hb_index=0)
    V = M.hybrid(V, tw, 1e7, 2, seed=1, cfg=0, hb_index=1)
    # near the minimum the action is quadratic in the 8 x 4V link deviations: (beta/3) s is at
    # most half their number (fewer, since gauge directions cost nothing), so s < 48 V / beta
    s = O.reduced_action(V, tw)
    Vol = 2 * 2 * 4 * 4
    assert 0 < s < 48 * Vol / 1e7
    assert s > 1e-2 * 48 * Vol / 1e7

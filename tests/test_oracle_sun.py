"""Pins of the oracle for SU(N), N != 3 (the l x l x Nl x Nl box with twist k, Sec. 1 and Sec. 5).

The oracle takes N from the field, so the SU(3) pins carry over; these fix what changes with N:
the centre factor exp(2 pi i k / N), the traceless projection 1/N, the plaquette normalisation
1/N, and the N x N exponential.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I

TW = I.default_twist(1)


def box(N, l=2):
    return (l, l, N * l, N * l)


@pytest.mark.parametrize("N,k", [(2, 1), (4, 1), (4, 3), (5, 2)])
def test_twist_eater_is_a_zero_action_stationary_point(N, k):
    L = box(N)
    U = I.twist_eater(L, k, N)
    tw = I.default_twist(k)
    assert abs(O.reduced_action(U, tw)) < 1e-12
    assert np.abs(O.force(U, tw)).max() < 1e-13
    m = O.measure(U, tw)
    assert abs(m["E"]) < 1e-14 and abs(m["Q"]) < 1e-14 and m["P"] == pytest.approx(1.0, abs=1e-14)
    # without the twist the same field has action: the twist factor is what cancels it
    assert O.reduced_action(U, np.zeros((4, 4), dtype=int)) > 0.1


@pytest.mark.parametrize("N", [2, 4])
def test_force_is_minus_twice_the_lie_derivative_of_s(N):
    L = (2, 2, 4, 4)
    U = I.random_links(L, 7, 0.5, N=N)
    Z = O.force(U, TW)
    T = I.sun_generators(N) * 0.5j  # anti-Hermitian, tr(T^a T^b) = -delta/2
    h = 1e-5
    for (x3, x2, x1, x0, mu) in [(0, 0, 0, 0, 0), (0, 0, 0, 0, 1), (1, 2, 1, 0, 2), (3, 3, 1, 1, 3), (0, 1, 0, 1, 1)]:
        for a in range(N * N - 1):
            def s_of(e):
                V = U.copy()
                V[x3, x2, x1, x0, mu] = scipy.linalg.expm(e * T[a]) @ U[x3, x2, x1, x0, mu]
                return O.reduced_action(V, TW)

            d = (s_of(h) - s_of(-h)) / (2 * h)
            za = -2 * np.trace(T[a] @ Z[x3, x2, x1, x0, mu]).real
            assert za == pytest.approx(-2 * d, abs=2e-6)
    assert np.abs(O.tr(Z)).max() < 1e-14 and np.abs(Z + O.dag(Z)).max() < 1e-14


@pytest.mark.parametrize("N", [2, 4])
def test_expm_matches_library(N):
    rng = np.random.default_rng(N)
    for scale in [1e-3, 0.3, 4.0]:
        A = rng.normal(size=(20, N, N)) + 1j * rng.normal(size=(20, N, N))
        X = scale * O.proj_ta(A)
        ref = np.array([scipy.linalg.expm(x) for x in X])
        assert np.abs(O.expm(X) - ref).max() < 1e-13 * max(1.0, scale)


@pytest.mark.parametrize("N", [2, 4])
def test_flow_keeps_sun_and_lowers_the_action(N):
    L = (2, 2, 4, 4)
    U = I.random_links(L, 11, 0.6, N=N)
    s0 = O.reduced_action(U, TW)
    V = O.rk3_step(U, 0.02, TW)
    assert O.reduced_action(V, TW) < s0
    assert np.abs(V @ O.dag(V) - np.eye(N)).max() < 1e-13
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-13


def test_rk3_is_third_order_su2():
    L = (2, 2, 4, 4)
    U = I.random_links(L, 3, 0.8, N=2)
    t = 0.16

    def run(eps):
        V = U
        for _ in range(int(round(t / eps))):
            V = O.rk3_step(V, eps, TW)
        return O.measure(V, TW)["E"]

    ref = run(0.000625)
    errs = [abs(run(e) - ref) for e in (0.01, 0.005)]
    assert errs[0] / errs[1] == pytest.approx(8.0, rel=0.1)


def _gauge(U, seed):
    L = O.extents_of(U)
    N = U.shape[-1]
    V = L[0] * L[1] * L[2] * L[3]
    Lam = I.random_sun(seed, V, 2.0, N).reshape(L[3], L[2], L[1], L[0], N, N)
    out = np.empty_like(U)
    for mu in range(4):
        Lp = np.roll(Lam, -1, axis=3 - mu)
        out[..., mu, :, :] = Lam @ U[..., mu, :, :] @ np.conj(np.swapaxes(Lp, -1, -2))
    return out


@pytest.mark.parametrize("N", [2, 4])
def test_observables_are_gauge_invariant(N):
    L = (2, 2, 4, 4)
    U = I.random_links(L, 5, 0.7, N=N)
    a, b = O.measure(U, TW), O.measure(_gauge(U, 9), TW)
    for key in "EQPS":
        assert b[key] == pytest.approx(a[key], rel=1e-11, abs=1e-12)


def test_su2_reflection_flips_q_and_keeps_e():
    # with the twist off, the reflection x3 -> -x3 of the links maps G to its mirror image:
    # E is unchanged and the epsilon-tensor sum of Q changes sign
    L = (4, 4, 4, 4)
    U = I.random_links(L, 2, 0.4, N=2)
    n0 = np.zeros((4, 4), dtype=int)
    m = O.measure(U, n0)
    R = U[(-np.arange(4)) % 4].copy()
    R[..., 3, :, :] = np.conj(np.swapaxes(U[(-np.arange(4) - 1) % 4][..., 3, :, :], -1, -2))
    r = O.measure(R, n0)
    assert m["E"] > 0
    assert r["E"] == pytest.approx(m["E"], rel=1e-12)
    assert r["Q"] == pytest.approx(-m["Q"], rel=1e-10, abs=1e-13)

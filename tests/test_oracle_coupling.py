"""Pins of the oracle's coupling normalisation (eqs. lambdat, calA, theta3, lambdat_latt, latt_norm)."""
import math

import numpy as np
import pytest

from oracle import tgf_oracle as O


@pytest.mark.parametrize("x", [0.05, 0.2827, 0.5, 1.0, 2.54, 9.0])
def test_theta3_two_series_agree(x):
    """eq. (theta3): the direct sum and the Poisson-resummed sum are the same function."""
    assert O.theta3_direct(x) == pytest.approx(O.theta3_dual(x), rel=1e-14)


def test_calA_small_x_limit():
    """theta3(0, ix) ~ x^-1/2 for x -> 0, so A(x) -> x^2 (1/x)(1/x - 1/(x N^2)) = 1 - 1/N^2."""
    assert O.calA(1e-3) == pytest.approx(1 - 1 / 9, rel=1e-12)


@pytest.mark.parametrize("c", [0.3, 0.4])
def test_lattice_norm_tends_to_continuum_with_a2_corrections(c):
    """N(c, Lt) -> 128 pi^2/(3 A(pi c^2)) as Lt -> oo, the gap shrinking ~4x per doubling of Lt."""
    cont = O.continuum_norm(c)
    gaps = [O.lattice_norm(c, Lt) / cont - 1 for Lt in (12, 24, 48)]
    assert abs(gaps[2]) < 2.5e-3
    assert 3.6 < gaps[0] / gaps[1] < 4.4 and 3.6 < gaps[1] / gaps[2] < 4.4


def test_lattice_norm_brute_force_tiny():
    """Literal quadruple loop over momenta for Lt = 6 against the vectorised sum."""
    c, Lt, N = 0.3, 6, 3
    tot = 0.0
    for n0 in range(Lt):
        for n1 in range(Lt):
            if n0 % N == 0 and n1 % N == 0:
                continue
            for n2 in range(Lt):
                for n3 in range(Lt):
                    q = [2 * math.pi * n / Lt for n in (n0, n1, n2, n3)]
                    qh2 = sum((2 * math.sin(x / 2)) ** 2 for x in q)
                    for mu in range(4):
                        for nu in range(4):
                            if mu != nu:
                                tot += math.exp(-0.25 * c * c * Lt * Lt * qh2) / qh2 * math.sin(q[nu]) ** 2 * math.cos(q[mu] / 2) ** 2
    assert O.lattice_norm_inverse(c, Lt) == pytest.approx(c ** 4 / 128 * tot, rel=1e-13)


def test_lambda_zero_charge_filter():
    E = [1.0, 2.0, 4.0, 8.0]
    Q = [0.1, -0.49, 0.5, -3.0]   # |Q| = 0.5 is excluded (strict <)
    lam, kept = O.lambda_tgf(0.3, 12, 0.5, E, Q)
    assert kept == 2
    assert lam == pytest.approx(O.lattice_norm(0.3, 12) * 0.25 * 1.5 / 3)
    assert O.lambda_tgf(0.3, 12, 0.5, [1.0], [2.0]) == (None, 0)

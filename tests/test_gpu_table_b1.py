"""End to end against numbers the paper prints: lambda_TGF at L~ = 12, 18b = 20 and 8 (Table B.1).

Ensembles are generated on the GPU (paper_2107_03747_gb300.ensemble) with the paper's hybrid
algorithm (tgf_mc_sweeps: one
heat-bath sweep and L~ over-relaxation sweeps per hybrid sweep, L~ hybrid sweeps between
measurements, Sec. 3.1), 256 independent chains started at the twist-eater (the classical
minimum of the twisted action).  Each measurement flows the configuration to sqrt(8t) = c L~
(c = 0.3, t = 1.62) in FP32 and takes the clover E and Q there; lambda_TGF = N(c, L~) t^2
<E d_Q> / (3 <d_Q>) (eq. lambdat_latt) with the lattice normalisation of eq. (latt_norm).
The statistical error is a jackknife over chains; the test accepts the printed value within
four combined standard deviations.  This pins, at once, the action and its twist factors, the
Monte Carlo weight, the flow, the clover energy density, the topological cut and N(c, L~).
"""
import math
import os

import numpy as np
import pytest


pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def printed(beta, Lt):
    for line in open(os.path.join(HERE, "golden", "table_b1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        b, l, lam, err = line.split()
        if float(b) == beta and int(l) == Lt:
            return float(lam), float(err)
    raise KeyError((beta, Lt))


@pytest.mark.parametrize("beta,therm", [(20.0, 50), (8.0, 150)])
def test_lambda_tgf_at_Lt12_matches_table_b1(tgf, beta, therm):
    from paper_2107_03747_gb300 import ensemble

    Lt, t, E, Q = ensemble.generate_and_measure(beta, l=4, chains=256, therm=therm, rounds=16, c=0.3, seed=2107)
    lam, err = ensemble.jackknife_lambda(0.3, Lt, t, E, Q)
    ref, ref_err = printed(beta, Lt)
    sigma = math.sqrt(err ** 2 + ref_err ** 2)
    half = [ensemble.jackknife_lambda(0.3, Lt, t, E[h::2], Q[h::2])[0] for h in (0, 1)]
    print(f"lambda_TGF(L~={Lt}, 18b={beta}): {lam:.5f} +- {err:.5f} (paper {ref} +- {ref_err}); "
          f"kept {int(np.sum(np.abs(Q) < 0.5))}/{Q.size}; {abs(lam - ref) / sigma:.2f} sigma; "
          f"even/odd rounds {half[0]:.5f} {half[1]:.5f}")
    assert err < 0.01 * lam
    assert abs(lam - ref) < 4 * sigma

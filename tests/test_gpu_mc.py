"""Parity of the Monte Carlo update on the GPU (tgf_mc_sweeps, through the C ABI) with the FP64
oracle of oracle/tgf_mc_oracle.py, link by link, on the same seeded fields and counter-based draws.

Bar: links within 1e-10 absolute after a few sweeps.  The two sides differ only in rounding (the
accept/reject decisions of the samplers are taken in FP64 on both sides), but the update
amplifies it: each heat-bath step divides by k, the norm of the SU(2) block of U Sigma (small
on disordered fields), and every pass feeds the links of the next; one FP64 rounding (1e-16)
grows to about 3e-12 over four link sweeps of a disordered 2x2x4x4 field.  The twisted action
agrees to 1e-11 relative.
"""
import numpy as np
import pytest

from oracle import tgf_mc_oracle as M
from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TW = I.default_twist(1)


def run_gpu(tgf, Ls, fields, beta, n_hybrid, n_or, seed, first):
    b = tgf.FlowBatch(Ls, "fp64", any_extents=True)
    b.set_links(fields)
    tgf.tgf_mc_sweeps(b.prec, b.lat, b.links, beta, n_hybrid, n_or, seed, first)
    return b.get_links()


def run_oracle(Ls, fields, beta, n_hybrid, n_or, seed, first):
    out = []
    for c, U in enumerate(fields):
        for h in range(n_hybrid):
            U = M.hybrid(U, TW, beta, n_or, seed, c, first + h)
        out.append(U)
    return out


@pytest.mark.parametrize("beta,n_or", [(5.0, 1), (0.7, 0)])
def test_mc_sweeps_match_oracle_small(tgf, beta, n_or):
    # beta = 5 takes the Kennedy-Pendleton branch, beta = 0.7 (disordered start) mostly Creutz's
    Ls = [(2, 2, 4, 4), (4, 2, 2, 6)]
    fields = [I.random_links(L, 40 + i, 0.9) for i, L in enumerate(Ls)]
    got = run_gpu(tgf, Ls, fields, beta, 2, n_or, 1234, 7)
    ref = run_oracle(Ls, fields, beta, 2, n_or, 1234, 7)
    for g, r, f in zip(got, ref, fields):
        assert np.abs(r - f).max() > 1e-2
        assert np.abs(g - r).max() <= 1e-10
        assert O.reduced_action(g, TW) == pytest.approx(O.reduced_action(r, TW), rel=1e-11)


def test_mc_sweeps_match_oracle_tgf_box(tgf):
    # the l = 4 box of the twisted gradient flow (L~ = 12) at 18 b = 20, from the twist-eater
    L = (4, 4, 12, 12)
    fields = [I.twist_eater(L, 1), I.random_links(L, 3, 0.3)]
    got = run_gpu(tgf, [L, L], fields, 20.0, 2, 3, 99, 0)
    ref = run_oracle([L, L], fields, 20.0, 2, 3, 99, 0)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-10
        s_g, s_r = O.reduced_action(g, TW), O.reduced_action(r, TW)
        assert s_g == pytest.approx(s_r, rel=1e-11)


def test_mc_sweeps_are_reproducible_and_seeded(tgf):
    L = (2, 2, 4, 4)
    f = [I.random_links(L, 5, 0.5)]
    a = run_gpu(tgf, [L], f, 3.0, 1, 1, 1, 0)[0]
    b = run_gpu(tgf, [L], f, 3.0, 1, 1, 1, 0)[0]
    c = run_gpu(tgf, [L], f, 3.0, 1, 1, 2, 0)[0]
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 1e-2

"""Parity of the SU(N) forms (tgf_sun_*, FP64, through the C ABI) with the oracle, N = 2, 3, 4.

Bar as for FP64 SU(3): 1e-12 relative on E, P, S, |dQ| <= 1e-12 max(1, |Q|), links 1e-12 absolute.
For N = 3 the SU(N) path is also checked against the SU(3) kernels on the same field.
"""
import numpy as np
import pytest

from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TW = I.default_twist(1)


def close(g, o, rel=1e-12):
    assert g[1] == pytest.approx(o["E"], rel=rel)
    assert abs(g[2] - o["Q"]) <= rel * max(1.0, abs(o["Q"]))
    assert g[3] == pytest.approx(o["P"], rel=rel)
    assert g[4] == pytest.approx(o["S"], rel=rel * 10, abs=rel * 100)


def fields_for(N):
    Ls = [(2, 2, 2 * N, 2 * N), (3, 2, 4, 5)]
    return Ls, [I.random_links(L, 60 + i + N, 0.6, N=N) for i, L in enumerate(Ls)]


@pytest.mark.parametrize("N", [2, 3, 4])
def test_sun_pack_roundtrip_and_measure(tgf, N):
    Ls, fs = fields_for(N)
    b = tgf.SunBatch(N, Ls, any_extents=True)
    b.set_links(fs)
    for f, g in zip(fs, b.get_links()):
        assert np.array_equal(f, g)
    got = b.measure(0.25)
    for i, f in enumerate(fs):
        assert got[i][0] == 0.25
        close(got[i], O.measure(f, TW))


@pytest.mark.parametrize("N", [2, 3, 4])
def test_sun_rk3_step_matches_oracle(tgf, N):
    Ls, fs = fields_for(N)
    b = tgf.SunBatch(N, Ls, any_extents=True)
    b.set_links(fs)
    b.step(0.02)
    b.step(0.02)
    got = b.measure(0.04)
    for i, (f, g) in enumerate(zip(fs, b.get_links())):
        ref = O.rk3_step(O.rk3_step(f, 0.02, TW), 0.02, TW)
        assert np.abs(g - ref).max() <= 1e-12
        close(got[i], O.measure(ref, TW))


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("eps", [0.2, 0.6])
def test_sun_large_steps_match_oracle(tgf, N, eps):
    # RK3 steps whose exponents exceed ||X||_F = 1/8, so the exponential scales by 2^-s and
    # squares back s >= 1 times; the oracle takes scipy's expm
    Ls, fs = fields_for(N)
    b = tgf.SunBatch(N, Ls, any_extents=True)
    b.set_links(fs)
    b.step(eps)
    for f, g in zip(fs, b.get_links()):
        ref = O.rk3_step(f, eps, TW)
        assert np.abs(g - ref).max() <= 1e-12


def test_sun3_agrees_with_the_su3_kernels(tgf):
    L = (4, 4, 12, 12)
    f = I.random_links(L, 8, 0.5)
    a = tgf.SunBatch(3, [L])
    a.set_links([f])
    s = tgf.FlowBatch([L], "fp64")
    s.set_links([f])
    ma, ms = a.measure(), s.measure()
    for k in range(1, 5):
        assert ma[0][k] == pytest.approx(ms[0][k], rel=1e-12, abs=1e-13)
    for _ in range(2):
        a.step(0.01)
        for st in (1, 2, 3):
            s.stage(st, 0.01)
    assert np.abs(a.get_links()[0] - s.get_links()[0]).max() <= 1e-13


@pytest.mark.parametrize("N,k", [(2, 1), (4, 1), (4, 3)])
def test_sun_twist_eater_is_static_on_the_nl_box(tgf, N, k):
    L = (2, 2, 2 * N, 2 * N)
    tw6 = (k, 0, 0, 0, 0, 0)
    b = tgf.SunBatch(N, [L], [tw6])
    U = I.twist_eater(L, k, N)
    b.set_links([U])
    m = b.measure()[0]
    assert abs(m[1]) < 1e-14 and abs(m[2]) < 1e-14 and m[3] == pytest.approx(1.0, abs=1e-14) and abs(m[4]) < 1e-12
    b.step(0.05)
    assert np.abs(b.get_links()[0] - U).max() < 1e-14


def test_sun_flow_on_the_nl_box_matches_oracle(tgf):
    # SU(2) on 4 x 4 x 8 x 8, a short flow with a measurement every step
    N, L = 2, (4, 4, 8, 8)
    f = I.random_links(L, 21, 0.5, N=N)
    b = tgf.SunBatch(N, [L])
    b.set_links([f])
    ref = f
    for step in range(5):
        close(b.measure(0.02 * step)[0], O.measure(ref, TW))
        b.step(0.02)
        ref = O.rk3_step(ref, 0.02, TW)
    assert np.abs(b.get_links()[0] - ref).max() <= 1e-12

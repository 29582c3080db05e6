"""The kernels' site indices on a self-checking build (-DTGF_CHECK, libtgf_check.so).

No memory checker can run on this GPU pool, so the library has a build in which every link,
accumulator and clover access checks its site index against the plane length and records a
violation instead of faulting.  This test runs the flow in every precision on mixed, ragged and
odd extents (with measurements every step), the standalone measurement and time slices, the
Monte Carlo update and the SU(N) forms on that build, in a child process, and requires that no
kernel recorded a violation.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
from paper_2107_03747_gb300 import binding as tgf
from paper_2107_03747_gb300 import inputs as I

assert tgf.LIB_PATH.endswith("libtgf_check.so"), tgf.LIB_PATH
Ls = [(4, 4, 12, 12), (3, 3, 5, 7), (2, 2, 6, 6), (6, 6, 18, 18), (5, 2, 3, 4)]
fields = [I.random_links(L, 10 + i, 0.5) for i, L in enumerate(Ls)]
for prec in ("fp64", "fp32", "fp32_r12"):
    b = tgf.FlowBatch(Ls, prec, any_extents=True)
    b.set_links(fields)
    b.flow(0.01, [0.03, 0.02, 0.05, 0.01, 0.025], measure_every=1)
    b.measure()
    b.slices(3)
    b.get_links()
    assert tgf.tgf_check_errors() == 0, prec
# every launch tile of the FP32 forms, on boxes with and without the hypercube order and with
# partly filled last blocks
from paper_2107_03747_gb300 import tune
Lt = [(4, 4, 12, 12), (3, 3, 5, 7), (8, 4, 6, 2), (6, 6, 18, 18)]
ft = [I.random_links(L, 30 + i, 0.5) for i, L in enumerate(Lt)]
for prec in ("fp32", "fp32_r12"):
    for tile in tune.TILES:
        b = tgf.FlowBatch(Lt, prec, any_extents=True)
        b.set_links(ft)
        b.flow(0.01, [0.03, 0.02, 0.04, 0.01], measure_every=2, flags=tune.tune_flags(1 if tile == 3 else 0, False, tile))
        assert tgf.tgf_check_errors() == 0, (prec, tile)
Lm = [(4, 4, 12, 12), (2, 2, 6, 6)]
m = tgf.FlowBatch(Lm, "fp64")
m.set_links([I.random_links(L, 3, 0.5) for L in Lm])
tgf.tgf_mc_sweeps(m.prec, m.lat, m.links, 6.0, 1, 2, 5, 0)
assert tgf.tgf_check_errors() == 0, "mc"
for N in (2, 3, 4):
    Ls2 = [(2, 2, 2 * N, 2 * N), (3, 2, 4, 5)]
    s = tgf.SunBatch(N, Ls2, any_extents=True)
    s.set_links([I.random_links(L, 1, 0.5, N=N) for L in Ls2])
    s.step(0.01)
    s.measure()
    s.get_links()
    assert tgf.tgf_check_errors() == 0, N
print("checked ok")
"""


def test_self_checking_build_records_no_violation(tgf):
    from paper_2107_03747_gb300 import build

    lib = build.build(check=True)
    env = dict(os.environ, TGF_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked ok" in r.stdout

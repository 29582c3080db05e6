"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element.

FP64 bar: 1e-12 relative on E, P, S; |dQ| <= 1e-12 max(1, |Q|); links 1e-12 absolute.
FP32 bars: the stated FP32 tolerances below (links ~1e-5 after a step, |dE/E| <= 1e-6 on the flow).
"""
import math
import os

import numpy as np
import pytest

from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I
from tests import fields as F

pytestmark = pytest.mark.gpu

TW = I.default_twist(1)
HERE = os.path.dirname(os.path.abspath(__file__))


def close_obs(g, o, rel=1e-12):
    """g: (t, E, Q, P, S) from the GPU; o: oracle dict or tuple."""
    if isinstance(o, dict):
        o = (g[0], o["E"], o["Q"], o["P"], o["S"])
    assert g[0] == pytest.approx(o[0], abs=1e-12)
    assert g[1] == pytest.approx(o[1], rel=rel, abs=1e-300)
    assert abs(g[2] - o[2]) <= rel * max(1.0, abs(o[2]))
    assert g[3] == pytest.approx(o[3], rel=rel)
    assert g[4] == pytest.approx(o[4], rel=rel * 10, abs=rel * 100)


def batch(tgf, Ls, prec="fp64", twists=None):
    return tgf.FlowBatch(Ls, prec, twists, any_extents=True)


def load(tgf, Ls, fields, prec="fp64", twists=None):
    b = batch(tgf, Ls, prec, twists)
    b.set_links(fields)
    return b


# ---- layout ------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_pack_unpack_roundtrip(tgf, prec):
    Ls = [(4, 4, 12, 12), (3, 3, 5, 7)]
    fields = [I.random_links(L, 20 + i, 0.7) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields, prec)
    back = b.get_links()
    for f, g in zip(fields, back):
        if prec == "fp64":
            assert np.array_equal(f, g)
        elif prec == "fp32":
            assert np.abs(f - g).max() <= 6e-8
        else:
            assert np.abs(f[..., :2, :] - g[..., :2, :]).max() <= 6e-8
            assert np.abs(f[..., 2, :] - g[..., 2, :]).max() <= 5e-7  # rebuilt from rounded rows


# ---- observables -------------------------------------------------------------------------------

def test_measure_matches_oracle_fp64(tgf):
    cases = [((4, 4, 12, 12), TW, 0), ((3, 3, 5, 7), TW, 1), ((2, 2, 6, 6), TW, 2)]
    # a twist in three planes (including a long one) exercises every twisted leaf position
    tw3 = np.zeros((4, 4), dtype=np.int64)
    for a, b_, k in [(0, 1, 1), (0, 2, 2), (1, 3, 1)]:
        tw3[a, b_], tw3[b_, a] = k, -k
    cases.append(((4, 3, 5, 6), tw3, 3))
    Ls = [c[0] for c in cases]
    fields = [I.random_links(L, s, 0.6) for L, _, s in cases]
    b = load(tgf, Ls, fields, "fp64", [tgf.twist6(c[1]) for c in cases])
    g = b.measure(t=0.25)
    for i, (L, tw, _) in enumerate(cases):
        o = O.measure(fields[i], tw)
        close_obs(g[i], o)
        assert g[i][0] == 0.25


def test_measure_traceless_flag(tgf):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 5, 0.5)
    b = load(tgf, [L], [U])
    g = b.measure(flags=tgf.TGF_CLOVER_TRACELESS)[0]
    close_obs(g, O.measure(U, TW, traceless=True))
    g0 = b.measure()[0]
    assert g0[1] != g[1]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_twist_eater_on_gpu(tgf, prec):
    L = (4, 4, 12, 12)
    b = load(tgf, [L], [I.twist_eater(L)], prec)
    g = b.measure()[0]
    tol = 1e-14 if prec == "fp64" else 1e-6
    assert abs(g[1]) < tol and abs(g[2]) < tol and abs(g[3] - 1) < tol
    # the eater is a fixed point of the flow
    obs, n = b.flow(0.05, 0.2)
    o = obs.cpu().numpy()[0, : n[0]]
    assert np.abs(o[:, 1]).max() < tol and np.abs(o[:, 3] - 1).max() < tol


def test_gauge_invariance_on_gpu(tgf):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 8, 0.5)
    Ug = F.gauge_transform(U, F.random_gauge(L, 77))
    b = load(tgf, [L, L], [U, Ug])
    g = b.measure()
    for k in range(1, 5):
        assert g[1][k] == pytest.approx(g[0][k], rel=1e-12, abs=1e-13)
    obs, n = b.flow(0.02, 0.1)
    o = obs.cpu().numpy()
    assert np.allclose(o[0, : n[0], 1:], o[1, : n[1], 1:], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp32_r12", 2e-6)])
def test_measure_fp32_forms(tgf, prec, tol):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 0, 0.3)
    g = load(tgf, [L], [U], prec).measure()[0]
    o = O.measure(U, TW)
    assert g[1] == pytest.approx(o["E"], rel=tol)
    assert abs(g[2] - o["Q"]) < tol * 10
    assert g[3] == pytest.approx(o["P"], rel=tol)


# ---- one RK3 step ------------------------------------------------------------------------------

def test_three_stages_equal_one_rk3_step_fp64(tgf):
    Ls = [(4, 4, 12, 12), (3, 3, 5, 7)]
    fields = [I.random_links(L, 30 + i, 0.5) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields)
    eps = 0.03
    for s in (1, 2, 3):
        b.stage(s, eps)
    got = b.get_links()
    for f, g in zip(fields, got):
        ref = O.rk3_step(f, eps, TW)
        assert np.abs(g - ref).max() < 1e-13


def test_stage_one_is_exp_quarter_force(tgf):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 31, 0.6)
    b = load(tgf, [L], [U])
    b.stage(1, 0.1)
    ref = np.matmul(O.expm(0.025 * O.force(U, TW)), U)
    assert np.abs(b.get_links()[0] - ref).max() < 1e-14


def test_large_step_uses_scaling_and_squaring(tgf):
    """eps Z with ||.||_F > 1 takes the scaled exponential path."""
    L = (2, 2, 6, 6)
    U = I.random_links(L, 32, 1.5)
    b = load(tgf, [L], [U])
    b.stage(1, 2.0)
    ref = np.matmul(O.expm(0.5 * O.force(U, TW)), U)
    assert np.abs(ref).max() > 0
    assert np.abs(b.get_links()[0] - ref).max() < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-6), ("fp32_r12", 3e-6)])
def test_rk3_step_fp32_forms(tgf, prec, tol):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 33, 0.5)
    b = load(tgf, [L], [U], prec)
    for s in (1, 2, 3):
        b.stage(s, 0.01, reunit=1 if s == 3 else 0)
    g = b.get_links()[0]
    ref = O.rk3_step(U, 0.01, TW)
    assert np.abs(g - ref).max() < tol
    assert np.abs(g @ O.dag(g) - np.eye(3)).max() < 1e-6


# ---- whole flows ---------------------------------------------------------------------------------

def read_golden(name):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", name)) if not l.startswith("#")]
    return np.array([[float(x) for x in r] for r in rows])


def test_flow_l4_matches_stored_oracle_trajectory(tgf):
    """4x4x12x12, seed 0, amp 0.3, eps 0.01 to t = 0.18: every record against the stored oracle run."""
    L = (4, 4, 12, 12)
    ref = read_golden("flow_l4_seed0.txt")
    b = load(tgf, [L], [I.random_links(L, 0, 0.3)])
    obs, n = b.flow(0.01, 0.18)
    o = obs.cpu().numpy()[0, : n[0]]
    assert n[0] == len(ref) == 19
    for g, r in zip(o, ref):
        close_obs(g, r)


def test_flow_final_links_match_oracle(tgf):
    L = (2, 2, 6, 6)
    U = I.random_links(L, 3, 0.5)
    ref = read_golden("flow_l2_seed3.txt")
    Uo, rec = O.flow(U, 0.02, 0.1, TW)
    b = load(tgf, [L], [U])
    obs, n = b.flow(0.02, 0.1)
    o = obs.cpu().numpy()[0, : n[0]]
    for g, r, r2 in zip(o, rec, ref):
        close_obs(g, r)
        close_obs(g, r2)
    assert np.abs(b.get_links()[0] - Uo).max() < 1e-12


def test_flow_mixed_batch_partial_steps_and_measure_every(tgf):
    """Configurations of different sizes and end times (one with a partial last step) in one flow."""
    Ls = [(2, 2, 6, 6), (3, 3, 9, 9), (4, 4, 12, 12), (2, 3, 4, 5)]
    tends = [0.05, 0.045, 0.03, 0.0]
    fields = [I.random_links(L, 40 + i, 0.5) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields)
    obs, n = b.flow(0.01, tends, measure_every=2)
    o = obs.cpu().numpy()
    finals = b.get_links()
    for i, (U, te) in enumerate(zip(fields, tends)):
        Uo, rec = O.flow(U, 0.01, te, TW, measure_every=2)
        assert n[i] == len(rec)
        for g, r in zip(o[i, : n[i]], rec):
            close_obs(g, r)
        assert np.abs(finals[i] - Uo).max() < 1e-12


def test_graph_and_direct_launches_agree_bitwise(tgf):
    Ls = [(4, 4, 12, 12), (2, 2, 6, 6)]
    fields = [I.random_links(L, 50 + i, 0.4) for i, L in enumerate(Ls)]
    res = []
    for flags in (0, tgf.TGF_NO_GRAPH, 0):
        b = load(tgf, Ls, fields)
        obs, n = b.flow(0.01, [0.07, 0.05], flags=flags)
        res.append((obs.cpu().numpy().copy(), [f.copy() for f in b.get_links()]))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0])
        for a, c in zip(r[1], res[0][1]):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", ["fp32", "fp32_r12"])
def test_flow_fp32_forms_energy_error(tgf, prec):
    """FP32 links with FP64 sums on the 4x4x12x12 flow: |dE/E| <= 1e-6 at every record."""
    L = (4, 4, 12, 12)
    ref = read_golden("flow_l4_seed0.txt")
    b = load(tgf, [L], [I.random_links(L, 0, 0.3)], prec)
    obs, n = b.flow(0.01, 0.18, reunit_every=1)
    o = obs.cpu().numpy()[0, : n[0]]
    rel = np.abs(o[:, 1] / ref[:, 1] - 1)
    assert rel.max() <= 1e-6, rel.max()
    assert np.abs(o[:, 2] - ref[:, 2]).max() < 1e-5


def test_flow_to_the_paper_scale_matches_stored_oracle_trajectory(tgf):
    """4x4x12x12 (L~ = 12) flowed to the coupling's own scale sqrt(8t) = 0.3 L~ (Sec. 3.1, eq.
    lambdat_latt), t = 1.62, 162 steps: FP64 against the stored oracle run at every record to 1e-12,
    and lambda_TGF of that record against the oracle's."""
    L = (4, 4, 12, 12)
    ref = read_golden("flow_l4_seed0_paper_scale.txt")
    b = load(tgf, [L], [I.random_links(L, 0, 0.3)])
    obs, n = b.flow(0.01, 1.62)
    o = obs.cpu().numpy()[0, : n[0]]
    assert n[0] == len(ref) == 163
    for g, r in zip(o, ref):
        close_obs(g, r)
    lam, kept = tgf.tgf_lambda(0.3, 12, 1.62, [o[-1, 1]], [o[-1, 2]])
    lo, ko = O.lambda_tgf(0.3, 12, 1.62, [ref[-1, 1]], [ref[-1, 2]])
    assert kept == ko == 1 and lam == pytest.approx(lo, rel=1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp32_r12"])
def test_fp32_forms_to_the_paper_scale_against_the_oracle(tgf, prec):
    """The FP32 forms over the same 162 steps with the bench's re-projection period (20 steps):
    |dE/E| <= 1e-6 at every record against the oracle (the configuration has |Q| < 1/2, so it is one
    lambda_TGF keeps), |dQ| <= 1e-5, P to 1e-6 and S to 1e-5 relative."""
    L = (4, 4, 12, 12)
    ref = read_golden("flow_l4_seed0_paper_scale.txt")
    b = load(tgf, [L], [I.random_links(L, 0, 0.3)], prec)
    obs, n = b.flow(0.01, 1.62, reunit_every=20)
    o = obs.cpu().numpy()[0, : n[0]]
    assert n[0] == len(ref)
    assert abs(ref[-1, 2]) < 0.5
    rel = np.abs(o[:, 1] / ref[:, 1] - 1)
    assert rel.max() <= 1e-6, rel.max()
    assert np.abs(o[:, 2] - ref[:, 2]).max() <= 1e-5
    assert np.abs(o[:, 3] / ref[:, 3] - 1).max() <= 1e-6
    assert np.abs(o[:, 4] / ref[:, 4] - 1).max() <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "fp32_r12"])
def test_fp32_forms_on_the_l6_ensemble_member_against_the_oracle(tgf, prec):
    """6x6x18x18 member of the mixed ensemble (seed 1) to t = c^2 l^2/8 = 0.405, 40 steps and one of
    0.005: the FP32 forms against the stored oracle trajectory at every record, |dE/E| <= 1e-6."""
    L = (6, 6, 18, 18)
    ref = read_golden("flow_l6_batched1.txt")
    _, U = I.batched_member(1, L)
    b = load(tgf, [L], [U], prec)
    obs, n = b.flow(0.01, 0.405, reunit_every=20)
    o = obs.cpu().numpy()[0, : n[0]]
    assert n[0] == len(ref) == 42
    assert o[:, 0] == pytest.approx(ref[:, 0], abs=1e-12)
    rel = np.abs(o[:, 1] / ref[:, 1] - 1)
    assert rel.max() <= 1e-6, rel.max()
    assert np.abs(o[:, 2] - ref[:, 2]).max() <= 1e-5
    assert np.abs(o[:, 3] / ref[:, 3] - 1).max() <= 1e-6
    assert np.abs(o[:, 4] / ref[:, 4] - 1).max() <= 1e-5


def test_flow_is_reproducible_bitwise(tgf):
    L = (4, 4, 12, 12)
    U = I.random_links(L, 9, 0.5)
    outs = []
    for _ in range(2):
        b = load(tgf, [L], [U], "fp32")
        obs, n = b.flow(0.01, 0.05)
        outs.append(obs.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_flow_records_equal_standalone_measurements_bitwise(tgf, prec):
    """A measured flow step takes the clover halves from its stage-1 launch (the stage kernel's
    mode 1), tgf_measure from a halves-only launch (mode 2); both then run the same sum and
    reduction.  The scalar arithmetic of the halves is written as explicit fma chains, so the
    two kernels round alike: every record of a flow equals tgf_measure of the field at that step
    bit for bit, for every launch tile but the shared-corner one and with the configurations
    reordered by size."""
    from paper_2107_03747_gb300 import tune

    Ls = [(4, 4, 12, 12), (3, 3, 9, 9), (2, 2, 6, 6)]
    fields = [I.random_links(L, 130 + i, 0.5) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields, prec)
    ref = [b.measure(0.0)]
    for k in range(3):  # fields after 1, 2, 3 steps, measured stand-alone
        b.flow(0.01, 0.01, measure_every=100)
        ref.append(b.measure(0.01 * (k + 1)))
    for f in tune.candidates(tgf.PRECISIONS[prec]):
        b = load(tgf, Ls, fields, prec)
        obs, n = b.flow(0.01, 0.03, flags=f)
        o = obs.cpu().numpy().reshape(len(Ls), -1, 5)
        assert list(n) == [4, 4, 4]
        if tune.flags_setting(f)["shared_corners"]:
            # tile 3 rounds the flowed fields differently; its first record is of the input field
            assert np.array_equal(o[:, 0], ref[0])
            continue
        for k in range(4):
            assert np.array_equal(o[:, k], ref[k]), (f, k)


# ---- full-size workloads -------------------------------------------------------------------------

def test_full_size_l16_measure_and_stage(tgf):
    """16x16x48x48 (589,824 sites): observables and a first RK3 stage on every link against the oracle."""
    L = (16, 16, 48, 48)
    U = I.random_links(L, 0, 0.4)
    b = load(tgf, [L], [U])
    close_obs(b.measure()[0], O.measure(U, TW))
    b.stage(1, 0.01)
    ref = np.matmul(O.expm(0.0025 * O.force(U, TW)), U)
    assert np.abs(b.get_links()[0] - ref).max() < 1e-14


def test_full_size_16_configs_l8_one_step_sampled(tgf):
    """16 configurations of 8x8x24x24 in one launch; configurations 0 and 13 checked link by link."""
    L = (8, 8, 24, 24)
    fields = [I.random_links(L, s, 0.3) for s in range(16)]
    b = load(tgf, [L] * 16, fields)
    g = b.measure()
    for s in (0, 13):
        close_obs(g[s], O.measure(fields[s], TW))
    for st in (1, 2, 3):
        b.stage(st, 0.01)
    got = b.get_links()
    for s in (0, 13):
        assert np.abs(got[s] - O.rk3_step(fields[s], 0.01, TW)).max() < 1e-13


def test_full_size_flow_properties_fp32(tgf):
    """l/a = 16 flowed in FP32 to t = 0.5: S falls monotonically, E falls, links stay in SU(3)."""
    L = (16, 16, 48, 48)
    U = I.random_links(L, 1, 0.4)
    b = load(tgf, [L], [U], "fp32")
    obs, n = b.flow(0.01, 0.5, reunit_every=10)
    o = obs.cpu().numpy()[0, : n[0]]
    assert np.all(np.diff(o[:, 4]) < 0)
    assert np.all(np.diff(o[:, 1]) < 0)
    g = b.get_links()[0]
    assert np.abs(g @ O.dag(g) - np.eye(3)).max() < 2e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_r12"])
def test_fp32_small_extents_and_twists_along_x3(tgf, prec):
    """FP32 forms on extents 2 and odd extents along x3, with twists in planes that contain x3
    (their twisted corners sit on the x3 = 0 and x3 = 1 slabs)."""
    tw = np.zeros((4, 4), dtype=np.int64)
    for a, b_, k in [(0, 1, 1), (0, 3, 1), (1, 3, 2), (2, 3, 1)]:
        tw[a, b_], tw[b_, a] = k, -k
    cases = [(2, 3, 4, 2), (3, 2, 2, 4), (4, 4, 4, 6), (3, 3, 5, 7)]
    fields = [I.random_links(L, 70 + i, 0.5) for i, L in enumerate(cases)]
    b = load(tgf, cases, fields, prec, [tgf.twist6(tw)] * len(cases))
    g = b.measure()
    for i, L in enumerate(cases):
        o = O.measure(fields[i], tw)
        assert g[i][1] == pytest.approx(o["E"], rel=2e-6)
        assert abs(g[i][2] - o["Q"]) < 2e-5
        assert g[i][3] == pytest.approx(o["P"], rel=2e-6)
    for s in (1, 2, 3):
        b.stage(s, 0.02)
    got = b.get_links()
    for i, L in enumerate(cases):
        ref = O.rk3_step(fields[i], 0.02, tw)
        assert np.abs(got[i] - ref).max() < 5e-6, (L, np.abs(got[i] - ref).max())
    obs, n = b.flow(0.02, 0.06)
    o = obs.cpu().numpy()
    for i, L in enumerate(cases):
        _, rec = O.flow(O.rk3_step(fields[i], 0.02, tw), 0.02, 0.06, tw)
        for gg, r in zip(o[i, : n[i]], rec):
            assert gg[1] == pytest.approx(r[1], rel=5e-6)


# ---- time-slice charge (Sec. 4) --------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_slice_charge_matches_oracle(tgf, prec, tol):
    Ls = [(4, 4, 12, 12), (3, 3, 5, 7)]
    fields = [I.random_links(L, 80 + i, 0.6) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields, prec)
    for direction in (3, 2, 0):
        got = b.slices(direction)
        for U, g in zip(fields, got):
            ref = O.slice_charge(U, TW, direction)
            scale = max(1.0, np.abs(ref).max())
            assert np.abs(g - ref).max() <= tol * scale, (direction, np.abs(g - ref).max())
    # slices add up to Q
    g = b.measure()
    for i, q in enumerate(b.slices(3)):
        assert q.sum() == pytest.approx(g[i][2], abs=tol * 10)


def test_slice_charge_full_size_l16_sums_to_q(tgf):
    L = (16, 16, 48, 48)
    U = I.random_links(L, 2, 0.4)
    b = load(tgf, [L], [U], "fp32")
    b.flow(0.01, 0.3)
    q = b.slices(3)[0]
    Q = b.measure()[0][2]
    assert q.shape == (48,)
    assert q.sum() == pytest.approx(Q, abs=1e-5)


# ---- host-buffer path and resumed flows -------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_upload_download_through_host_buffers(tgf, prec):
    """tgf_upload / tgf_download move canonical host fields through a device staging buffer."""
    import torch

    Ls = [(4, 4, 12, 12), (3, 3, 5, 7), (2, 2, 6, 6)]
    fields = [I.random_links(L, 90 + i, 0.5) for i, L in enumerate(Ls)]
    host = torch.from_numpy(np.concatenate([f.view(np.float64).reshape(-1) for f in fields])).pin_memory()
    b = tgf.FlowBatch(Ls, prec, any_extents=True)
    staging = torch.empty(max(L[0] * L[1] * L[2] * L[3] for L in Ls) * 72, dtype=torch.float64, device="cuda")
    tgf.tgf_upload(b.prec, b.lat, host, staging, b.links)
    ref = b.get_links()
    out = torch.zeros_like(host).pin_memory()
    tgf.tgf_download(b.prec, b.lat, b.links, staging, out)
    flat = out.numpy()
    off = 0
    for L, r, f in zip(Ls, ref, fields):
        n = L[0] * L[1] * L[2] * L[3] * 72
        got = flat[off:off + n].view(np.complex128).reshape(r.shape)
        assert np.array_equal(got, r)
        if prec == "fp64":
            assert np.array_equal(got, f)
        off += n
    small = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(tgf.TgfError):
        tgf.tgf_upload(b.prec, b.lat, host, small, b.links)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resumed_flow_is_bitwise_identical(tgf, prec):
    """Flowing to t1 and then, from the resulting field, for t2 - t1 reproduces one flow to t2 (no
    re-projection scheduled): the state of the flow between steps is the field alone."""
    L = (4, 4, 12, 12)
    U = I.random_links(L, 95, 0.5)
    a = load(tgf, [L], [U], prec)
    oa, na = a.flow(0.01, 0.10)
    b = load(tgf, [L], [U], prec)
    ob1, nb1 = b.flow(0.01, 0.04)
    ob2, nb2 = b.flow(0.01, 0.06)
    assert np.array_equal(a.get_links()[0], b.get_links()[0])
    ra = oa.cpu().numpy()[0, : na[0]]
    rb = np.concatenate([ob1.cpu().numpy()[0, : nb1[0] - 1], ob2.cpu().numpy()[0, : nb2[0]]])
    assert np.array_equal(ra[:, 1:], rb[:, 1:])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_is_bitwise_identical(tgf, prec, tmp_path):
    """tgf_save at t = 0.04, tgf_load into a fresh batch, flow on: the same field as one flow to t = 0.10.
    The file is also parsed here from the format description (header, lattice, data, zlib CRC-32)."""
    import struct
    import zlib

    import torch

    L = (4, 4, 12, 12)
    U = I.random_links(L, 97, 0.5)
    a = load(tgf, [L], [U], prec)
    a.flow(0.01, 0.10)
    b = load(tgf, [L], [U], prec)
    b.flow(0.01, 0.04)
    staging = torch.empty(L[0] * L[1] * L[2] * L[3] * 72, dtype=torch.float64, device="cuda")
    path = tmp_path / "mid.tgf"
    tgf.tgf_save(path, b.prec, b.lat, b.links, staging, 0.04, 4, 1234)
    raw = path.read_bytes()
    assert zlib.crc32(raw[:-4]) == struct.unpack("<I", raw[-4:])[0]
    magic, ver, ncfg, p, _, t, step, seed = struct.unpack("<8sIIiidqQ", raw[:48])
    assert (magic, ver, ncfg, t, step, seed) == (b"TGFCKPT1", 1, 1, 0.04, 4, 1234)
    assert struct.unpack("<4i6i", raw[48:88]) == (*L, 1, 0, 0, 0, 0, 0)
    data = np.frombuffer(raw[88:-4], dtype=np.complex128).reshape(U.shape)
    assert np.array_equal(data, b.get_links()[0])
    c = tgf.FlowBatch([L], prec)
    assert tgf.tgf_load(path, c.prec, c.lat, c.links, staging) == (0.04, 4, 1234)
    assert np.array_equal(c.get_links()[0], b.get_links()[0])
    c.flow(0.01, 0.06)
    assert np.array_equal(a.get_links()[0], c.get_links()[0])


@pytest.mark.parametrize("prec", ["fp32", "fp32_r12", "fp64"])
def test_launch_tuning_settings_give_identical_flows(tgf, prec, tmp_path):
    """Every launch setting of the tuner (persistent grids, configurations by size) computes the
    same flow bit for bit; the tuner returns one of them and caches it."""
    from paper_2107_03747_gb300 import tune

    Ls = [(4, 4, 12, 12), (6, 6, 18, 18), (2, 2, 6, 6), (4, 4, 12, 12)]
    fields = [I.random_links(L, 70 + i, 0.5) for i, L in enumerate(Ls)]
    t_end = [0.05, 0.03, 0.04, 0.05]
    ref = None
    for f in tune.candidates(tgf.PRECISIONS[prec]):
        b = load(tgf, Ls, fields, prec)
        obs, nrec = b.flow(0.01, t_end, flags=f)
        got = (b.get_links(), obs.cpu().numpy(), list(nrec))
        if ref is None:
            ref = got
            continue
        assert ref[2] == got[2]
        if tune.flags_setting(f)["shared_corners"]:
            # tile 3 forms half the forward staples as (Z T_ba)^+ U^+: equal up to FP32 rounding
            assert all(np.abs(x - y).max() < 2e-6 for x, y in zip(ref[0], got[0]))
            assert np.allclose(ref[1], got[1], rtol=2e-6, atol=2e-6)
        else:
            assert all(np.array_equal(x, y) for x, y in zip(ref[0], got[0]))
            assert np.array_equal(ref[1], got[1])
    b = load(tgf, Ls, fields, prec)
    best = tune.tune(b, eps=0.01, steps=3, path=str(tmp_path / "tune.json"))
    assert best in tune.candidates(tgf.PRECISIONS[prec])
    assert all(np.array_equal(x, y) for x, y in zip(b.get_links(), fields)) or prec != "fp64"


@pytest.mark.parametrize("tile", [2, 3, 4])
@pytest.mark.parametrize("prec", ["fp32", "fp32_r12"])
def test_launch_tiles_match_the_oracle(tgf, prec, tile):
    """Tiles 2-4 (hypercube site order; forward-staple corners passed between direction warps
    through shared memory; a tighter register cap) on ragged boxes, some with a last block partly
    past the configuration's end (those lanes take part in the named barriers on site 0), some
    with the hypercube order (4x4x12x12, 8x4x6x2) and some without, twists in three planes: one
    RK3 step against the oracle on every link, and a short flow against the oracle's records."""
    from paper_2107_03747_gb300 import tune

    tw = np.zeros((4, 4), dtype=np.int64)
    for a, b_, k in [(0, 1, 1), (0, 3, 2), (1, 2, 1)]:
        tw[a, b_], tw[b_, a] = k, -k
    Ls = [(3, 3, 5, 7), (4, 4, 12, 12), (2, 3, 4, 5), (6, 6, 18, 18), (8, 4, 6, 2)]
    fields = [I.random_links(L, 400 + i, 0.5) for i, L in enumerate(Ls)]
    flags = tune.tune_flags(0, False, tile)
    b = load(tgf, Ls, fields, prec, [tgf.twist6(tw)] * len(Ls))
    obs, n = b.flow(0.02, 0.02, flags=flags)  # one step, no re-projection
    got = b.get_links()
    for i, U in enumerate(fields):
        ref = O.rk3_step(U, 0.02, tw)
        assert np.abs(got[i] - ref).max() < 5e-6, (Ls[i], np.abs(got[i] - ref).max())
    b = load(tgf, Ls, fields, prec, [tgf.twist6(tw)] * len(Ls))
    obs, n = b.flow(0.02, 0.08, flags=flags)
    o = obs.cpu().numpy()
    for i, U in enumerate(fields):
        _, rec = O.flow(U, 0.02, 0.08, tw)
        assert n[i] == len(rec)
        for g, r in zip(o[i, : n[i]], rec):
            assert g[1] == pytest.approx(r[1], rel=5e-6)
            assert abs(g[2] - r[2]) < 2e-5


def test_large_batch_uses_the_full_descriptor_and_matches_oracle(tgf):
    """More than 16 configurations take the 256-entry launch descriptor; 40 small mixed
    configurations, one RK3 step and a measurement each, against the oracle."""
    Ls = [(2, 2, 6, 6) if i % 3 else (4, 4, 12, 12) for i in range(40)]
    fields = [I.random_links(L, 300 + i, 0.6) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields, "fp64")
    for st in (1, 2, 3):
        b.stage(st, 0.02)
    got = b.get_links()
    m = b.measure(0.02)
    for i in range(len(Ls)):
        ref = O.rk3_step(fields[i], 0.02, TW)
        assert np.abs(got[i] - ref).max() <= 1e-12
        close_obs(m[i], O.measure(ref, TW))


def test_a_full_256_configuration_batch_flows_like_the_oracle(tgf):
    """The largest batch, TGF_MAX_CFG = 256 configurations of three box sizes and end times in one
    FP32 flow (one CUDA graph): four of them, one per size and the last, against the oracle."""
    Ls = [[(2, 2, 6, 6), (4, 4, 12, 12), (3, 3, 9, 9)][i % 3] for i in range(tgf.TGF_MAX_CFG)]
    t_end = [[0.03, 0.02, 0.025][i % 3] for i in range(tgf.TGF_MAX_CFG)]
    fields = [I.random_links(L, 500 + i, 0.4) for i, L in enumerate(Ls)]
    b = load(tgf, Ls, fields, "fp32")
    obs, n = b.flow(0.01, t_end)
    o = obs.cpu().numpy()
    for i in (0, 1, 2, tgf.TGF_MAX_CFG - 1):
        _, rec = O.flow(fields[i], 0.01, t_end[i], TW)
        assert n[i] == len(rec)
        for g, r in zip(o[i, : n[i]], rec):
            assert g[1] == pytest.approx(r[1], rel=2e-6)
            assert abs(g[2] - r[2]) < 2e-5

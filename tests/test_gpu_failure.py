"""Failure handling and the library-owned context on the GPU.

Faults are made on the host only (TGF_FAULT): a NaN planted in the device copy of an uploaded
field, an allocation refused before cudaMalloc, an argument check that fails.  Nothing faults,
traps or hangs on the device; every test checks that the GPU still computes the right flow
afterwards.
"""
import os

import numpy as np
import pytest
import torch

from oracle import tgf_oracle as O
from paper_2107_03747_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TW = I.default_twist(1)
L4 = (4, 4, 12, 12)


def golden(name):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", name)) if not l.startswith("#")]
    return np.array([[float(x) for x in r] for r in rows])


def flows_like_the_oracle(tgf, prec="fp64"):
    """A fresh 4x4x12x12 flow to t = 0.18 against the stored oracle trajectory (the GPU still works)."""
    ref = golden("flow_l4_seed0.txt")
    b = tgf.FlowBatch([L4], prec)
    b.set_links([I.random_links(L4, 0, 0.3)])
    obs, n = b.flow(0.01, 0.18, flags=tgf.TGF_SYNC)
    o = obs.cpu().numpy()[0, : n[0]]
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.abs(o[:, 1] / ref[:, 1] - 1).max() <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_in_an_uploaded_field_is_reported_as_ekernel(tgf, prec, monkeypatch):
    b = tgf.FlowBatch([L4, L4], prec)
    fields = [I.random_links(L4, 0, 0.3), I.random_links(L4, 1, 0.3)]
    host = torch.from_numpy(np.concatenate([f.view(np.float64).reshape(-1) for f in fields])).pin_memory()
    staging = torch.empty(L4[0] * L4[1] * L4[2] * L4[3] * 72, dtype=torch.float64, device="cuda")
    tgf.tgf_kernel_status()  # clear any earlier note
    monkeypatch.setenv("TGF_FAULT", "nan")
    tgf.tgf_upload(b.prec, b.lat, host, staging, b.links)
    monkeypatch.delenv("TGF_FAULT")
    assert np.isfinite(host.numpy()).all()  # the caller's buffer is untouched
    with pytest.raises(tgf.TgfError) as e:
        b.flow(0.01, 0.05, flags=tgf.TGF_SYNC)
    assert e.value.status == tgf.TGF_EKERNEL
    assert "configuration 0" in str(e.value)
    # the note is cleared by the report; the second configuration flowed normally
    tgf.tgf_kernel_status()
    flows_like_the_oracle(tgf, prec)


def test_measure_sync_and_kernel_status(tgf, monkeypatch):
    b = tgf.FlowBatch([L4], "fp64")
    U = I.random_links(L4, 2, 0.4)
    host = torch.from_numpy(U.view(np.float64).reshape(-1).copy()).pin_memory()
    staging = torch.empty(host.numel(), dtype=torch.float64, device="cuda")
    obs = torch.zeros(5, dtype=torch.float64, device="cuda")
    tgf.tgf_kernel_status()
    monkeypatch.setenv("TGF_FAULT", "nan")
    tgf.tgf_upload(b.prec, b.lat, host, staging, b.links)
    monkeypatch.delenv("TGF_FAULT")
    tgf.tgf_measure(b.prec, b.lat, b.links, b.scratch, obs, 1, 0, 0.0)  # no TGF_SYNC: nothing reported yet
    with pytest.raises(tgf.TgfError) as e:
        tgf.tgf_kernel_status()
    assert e.value.status == tgf.TGF_EKERNEL
    tgf.tgf_kernel_status()  # reported once, then cleared
    tgf.tgf_upload(b.prec, b.lat, host, staging, b.links)
    tgf.tgf_measure(b.prec, b.lat, b.links, b.scratch, obs, 1, 0, 0.0, tgf.TGF_SYNC)
    o = O.measure(U, TW)
    assert obs.cpu().numpy()[1] == pytest.approx(o["E"], rel=1e-12)


def test_injected_bad_argument_on_the_gpu(tgf, monkeypatch):
    b = tgf.FlowBatch([L4], "fp32")
    b.set_links([I.random_links(L4, 0, 0.3)])
    monkeypatch.setenv("TGF_FAULT", "badarg")
    with pytest.raises(tgf.TgfError) as e:
        b.flow(0.01, 0.05)
    assert e.value.status == tgf.TGF_EINVAL
    monkeypatch.delenv("TGF_FAULT")
    flows_like_the_oracle(tgf, "fp32")


def test_context_refuses_an_allocation_beyond_the_device(tgf):
    """Three 72x72x216x216 FP64 configurations need 418 GB of links: cudaMalloc refuses, tgf_create
    returns TGF_ENOMEM and leaves nothing allocated."""
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(tgf.TgfError) as e:
        tgf.Context([(72, 72, 216, 216)] * 3, "fp64")
    assert e.value.status == tgf.TGF_ENOMEM
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    flows_like_the_oracle(tgf)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_context_flow_matches_the_oracle(tgf, prec, tmp_path):
    """tgf_create / tgf_set_links / tgf_ctx_flow / tgf_get_links / tgf_ctx_measure / save / load /
    tgf_destroy on a ragged two-configuration batch against the oracle."""
    Ls = [L4, (3, 3, 5, 7)]
    fields = [I.random_links(L, 30 + i, 0.5) for i, L in enumerate(Ls)]
    ctx = tgf.Context(Ls, prec, reunit_every=0, any_extents=True)
    for i, f in enumerate(fields):
        ctx.set_links(i, f)
    m = ctx.measure(0.0)
    tol = 1e-12 if prec == "fp64" else 2e-6
    for i, f in enumerate(fields):
        o = O.measure(f, TW)
        assert m[i][1] == pytest.approx(o["E"], rel=tol)
        assert m[i][3] == pytest.approx(o["P"], rel=tol)
    rec, nw = ctx.flow(0.01, [0.05, 0.03])
    for i, (f, te) in enumerate(zip(fields, [0.05, 0.03])):
        Uo, ro = O.flow(f, 0.01, te, TW)
        assert nw[i] == len(ro)
        for g, r in zip(rec[i, : nw[i]], ro):
            assert g[1] == pytest.approx(r[1], rel=tol * 5)
        got = ctx.get_links(i)
        assert np.abs(got - Uo).max() <= (1e-12 if prec == "fp64" else 5e-6)
    path = tmp_path / "ctx.tgf"
    ctx.save(path, 0.05, 5, 11)
    before = [ctx.get_links(i) for i in range(2)]
    ctx.set_links(0, fields[0])
    assert ctx.load(path) == (0.05, 5, 11)
    assert all(np.array_equal(a, ctx.get_links(i)) for i, a in enumerate(before))
    ctx.close()


def test_context_reports_a_nan_field(tgf, monkeypatch):
    ctx = tgf.Context([L4], "fp32")
    monkeypatch.setenv("TGF_FAULT", "nan")
    ctx.set_links(0, I.random_links(L4, 0, 0.3))
    monkeypatch.delenv("TGF_FAULT")
    with pytest.raises(tgf.TgfError) as e:
        ctx.flow(0.01, 0.03)
    assert e.value.status == tgf.TGF_EKERNEL
    ctx.set_links(0, I.random_links(L4, 0, 0.3))
    rec, nw = ctx.flow(0.01, 0.18)
    ref = golden("flow_l4_seed0.txt")
    assert np.abs(rec[0, : nw[0], 1] / ref[:, 1] - 1).max() <= 1e-6
    ctx.close()

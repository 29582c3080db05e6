"""tgf_measure_noalloc: the measurement for callers that cannot allocate device memory.

Some callers may not call cudaMalloc at all -- a plug-in whose host application owns every
byte of device memory and hands it only input and output buffers, or a latency-critical loop
that cannot afford cudaMalloc's implicit device synchronisation.  For them the library keeps
the measurement's scratch in a fixed device array of its own.  These tests call that entry
point through the C ABI and check it against tgf_measure with caller-provided scratch, twice in
a row on different fields (the shared array keeps the previous call's contents), and check that
a batch too large for the array is refused with a message.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2107_03747_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_r12"])
def test_noalloc_matches_caller_scratch_twice_in_a_row(tgf, prec):
    Ls = [(4, 4, 12, 12), (3, 3, 5, 7)]
    fields = [[I.random_links(L, 60 + i + 10 * r, 0.5) for i, L in enumerate(Ls)] for r in range(2)]
    rel = 1e-12 if prec == "fp64" else 1e-6
    for r in range(2):
        b = tgf.FlowBatch(Ls, prec, any_extents=True)
        b.set_links(fields[r])
        ref = b.measure(t=0.125)  # tgf_measure, scratch from the caller
        obs = torch.full((len(Ls) * 5,), float("nan"), dtype=torch.float64, device="cuda")
        tgf.tgf_measure_noalloc(b.prec, b.lat, b.links, obs, 1, 0, 0.125)
        got = obs.cpu().numpy().reshape(len(Ls), 5)
        assert np.all(np.isfinite(got))
        assert got[:, 0] == pytest.approx(ref[:, 0])
        for k in (1, 3, 4):
            assert got[:, k] == pytest.approx(ref[:, k], rel=rel)
        assert np.abs(got[:, 2] - ref[:, 2]).max() <= rel * max(1.0, np.abs(ref[:, 2]).max())


def test_noalloc_rejects_a_batch_beyond_its_fixed_scratch(tgf):
    lat = tgf.lattices([(16, 16, 48, 48)])
    links = torch.empty(256, dtype=torch.uint8, device="cuda")
    obs = torch.empty(5, dtype=torch.float64, device="cuda")
    with pytest.raises(tgf.TgfError) as e:
        tgf.tgf_measure_noalloc(tgf.TGF_FP64, lat, links, obs, 1, 0, 0.0)
    assert e.value.status == tgf.TGF_EINVAL
    assert "scratch" in str(e.value)

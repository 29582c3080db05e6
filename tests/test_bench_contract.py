"""bench.py's reference arm (the oracle on the host) prints the contract's JSON line; no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "l4", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "flowed site-RK3-steps/s" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["higher_is_better"] is True and d["vs_baseline"] is None


def test_reference_arm_on_other_ranks_prints_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "l4", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_stage_timing_runs_the_stages_in_rk3_order(monkeypatch):
    """time_stages launches stages 1, 2, 3 in order per repetition (so every stage sees the
    accumulator X of a real step) and times each stage between the events around its launch;
    checked with fake events and a fake library on the host."""
    import itertools
    import types

    import torch

    sys.path.insert(0, ROOT)
    import bench

    clock = itertools.count()

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = None

        def record(self, stream=None):
            self.t = next(clock)

        def elapsed_time(self, other):
            return float(other.t - self.t)

    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    calls = []

    def stage(prec, lat, w_in, w_out, accum, s, eps, reunit, flags):
        calls.append(s)
        assert (w_in, w_out, reunit, flags) == ("links", "tmp", 0, 3 << 13)
        next(clock)  # a stage takes one tick between its events

    tgf = types.SimpleNamespace(tgf_stage=stage, tgf_measure=lambda *a: next(clock))
    b = types.SimpleNamespace(prec=1, lat=None, links="links", links_tmp="tmp", accum=None, scratch=None, ncfg=1,
                              device="cpu")
    stage_ms, meas_ms = bench.time_stages(tgf, b, "fp32", nrep=4, flags=(3 << 13) | (1 << 12))
    assert calls == [1, 2, 3] * 5  # one warm-up step, then 4 timed ones
    assert stage_ms == [2.0, 2.0, 2.0] and meas_ms > 0

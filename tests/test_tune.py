"""The launch tuner's host logic: workload keys, the choice, the cache (no GPU: a fake timer)."""
import json

from paper_2107_03747_gb300 import tune


class FakeBatch:
    def __init__(self, prec, Ls):
        self.prec, self.Ls = prec, Ls


def test_candidates_cover_the_default_and_every_setting():
    c = tune.candidates(1)
    assert 0 in c and len(set(c)) == len(tune.GRIDS) * len(tune.ORDERS) * len(tune.TILES)
    c64 = tune.candidates(0)
    assert 0 in c64 and len(set(c64)) == len(tune.GRIDS) * len(tune.ORDERS)
    assert all((f >> 13) & 3 == 0 for f in c64)  # FP64 has one tile
    assert tune.tune_flags(2, True) == (2 << 8) | (1 << 12)
    assert tune.tune_flags(1, False, 2) == (1 << 8) | (2 << 13)
    assert tune.tune_flags(0, False, 4) == 4 << 13
    assert tune.flags_setting(tune.tune_flags(1, True, 1)) == {
        "grid_k": 1, "size_order": True, "tile": 1, "sites_per_block": 64, "resident_blocks_per_sm": 2,
        "site_order": "consecutive", "shared_corners": False}
    assert tune.flags_setting(tune.tune_flags(0, False, 3))["shared_corners"]
    assert tune.flags_setting(tune.tune_flags(0, False, 2))["site_order"] == "4x2x2x2 hypercube"
    s4 = tune.flags_setting(tune.tune_flags(0, False, 4))
    assert not s4["shared_corners"] and s4["resident_blocks_per_sm"] == 5


def test_workload_key_ignores_member_order():
    a = tune.workload_key(1, [(4, 4, 12, 12), (8, 8, 24, 24), (4, 4, 12, 12)], 1)
    b = tune.workload_key(1, [(8, 8, 24, 24), (4, 4, 12, 12), (4, 4, 12, 12)], 1)
    assert a == b
    assert a != tune.workload_key(0, [(4, 4, 12, 12), (8, 8, 24, 24), (4, 4, 12, 12)], 1)
    assert a != tune.workload_key(1, [(4, 4, 12, 12), (8, 8, 24, 24)], 1)


def test_choice_and_ties():
    assert tune.choose({0: 2.0, 256: 1.5, 4096: 1.7}) == 256
    assert tune.choose({4096: 1.0, 0: 1.0, 256: 1.0}) == 0


def test_tune_stores_and_reuses_the_winner(tmp_path):
    path = str(tmp_path / "t.json")
    calls = []

    def timer(flags):
        calls.append(flags)
        return 1.0 if flags == tune.tune_flags(2, True) else 2.0

    b = FakeBatch(1, [(8, 8, 24, 24)] * 16)
    best = tune.tune(b, path=path, timer=timer)
    assert best == tune.tune_flags(2, True)
    assert sorted(calls) == sorted(tune.candidates(1))
    d = json.load(open(path))
    assert list(d.values())[0]["flags"] == best
    calls.clear()
    assert tune.tune(b, path=path, timer=timer) == best and calls == []  # cache hit
    assert tune.tune(b, path=path, timer=lambda f: 1.0, force=True) == 0  # re-timed: ties go to the default

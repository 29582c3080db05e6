"""Launch tuner of tgf_flow: times the launch settings on the actual workload and caches the winner.

The settings (tgf.h: TGF_TUNE_GRID(k), TGF_TUNE_SIZE_ORDER, TGF_TUNE_TILE(t)) change how the
stage kernels are scheduled, never what they compute: the launch tile of the FP32 forms (32 or 64
sites per block, and the register cap that sets how many blocks share an SM), a persistent grid
of k x SMs x resident blocks that loops over the tiles (k = 0: one block per tile), and the order
of the configurations inside each launch (as given, or largest first).  For a workload -- precision, the multiset of
extents, measurement interval -- the tuner flows the batch for a few steps under every
candidate (each captured as its own CUDA graph), times the best of `reps` replays with CUDA
events, and stores the fastest flags in a JSON cache (path from TGF_TUNE_CACHE, else
~/.cache/tgf/tune.json).  Later calls with the same workload read the cache.
"""
from __future__ import annotations

import json
import os
from collections import Counter

GRIDS = (0, 1, 2, 4)
ORDERS = (False, True)
# launch tiles of the FP32 forms' stage kernels (tgf.h TGF_TUNE_TILE): 32 consecutive sites per
# block, 64 sites per block (two warps per direction), 32 sites as a 4x2x2x2 hypercube, the first
# with the forward-staple corners shared in pairs of direction warps, the first with 5 blocks per SM
TILES = (0, 1, 2, 3, 4)
TGF_TUNE_SIZE_ORDER = 1 << 12
TGF_FP64 = 0


def tune_flags(grid: int, by_size: bool, tile: int = 0) -> int:
    return ((grid & 0xF) << 8) | (TGF_TUNE_SIZE_ORDER if by_size else 0) | ((tile & 0x7) << 13)


def flags_setting(flags: int) -> dict:
    """The launch setting a flags word selects (reported next to bench numbers)."""
    tile = (flags >> 13) & 0x7
    return {"grid_k": (flags >> 8) & 0xF, "size_order": bool(flags & TGF_TUNE_SIZE_ORDER), "tile": tile,
            "sites_per_block": 64 if tile == 1 else 32,
            "resident_blocks_per_sm": 2 if tile == 1 else 5 if tile == 4 else 4,
            "site_order": "4x2x2x2 hypercube" if tile == 2 else "consecutive",
            "shared_corners": tile == 3}


def candidates(prec: int | None = None):
    """Every setting of the search space; FP64 has the default tile only."""
    tiles = (0,) if prec == TGF_FP64 else TILES
    return [tune_flags(g, o, t) for t in tiles for g in GRIDS for o in ORDERS]


def workload_key(prec: int, Ls, measure_every: int) -> str:
    ext = sorted(Counter(tuple(int(x) for x in L) for L in Ls).items())
    return json.dumps({"prec": int(prec), "extents": [[list(e), n] for e, n in ext], "measure_every": int(measure_every)},
                      sort_keys=True)


def cache_path() -> str:
    return os.environ.get("TGF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "tgf", "tune.json"))


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(times: dict) -> int:
    """The fastest candidate; ties go to the simplest (smaller flag value)."""
    return min(sorted(times), key=lambda f: times[f])


def tune(batch, eps: float = 0.01, steps: int = 4, measure_every: int = 1, reps: int = 3, path: str | None = None,
         timer=None, force: bool = False) -> int:
    """Best tgf_flow flags for `batch` (a binding.FlowBatch); the batch's fields are restored afterwards.

    `timer(flags) -> ms` replaces the GPU timing (tests on the host)."""
    key = workload_key(batch.prec, batch.Ls, measure_every)
    if not force:
        hit = load_cache(path).get(key)
        if hit is not None:
            return int(hit["flags"])
    if timer is None:
        timer = _gpu_timer(batch, eps, steps, measure_every, reps)
    times = {f: float(timer(f)) for f in candidates(batch.prec)}
    best = choose(times)
    store(key, {"flags": best, "ms": {str(f): t for f, t in times.items()}, "steps": steps}, path)
    return best


def _gpu_timer(batch, eps, steps, measure_every, reps):
    import torch

    saved = batch.links.clone()
    t_end = eps * steps

    def run(flags):
        best = float("inf")
        for r in range(reps + 1):
            batch.links.copy_(saved)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            batch.flow(eps, t_end, measure_every=measure_every, flags=flags)
            b.record()
            torch.cuda.synchronize()
            if r:  # the first run captures the graph
                best = min(best, a.elapsed_time(b))
        batch.links.copy_(saved)
        return best

    return run

"""Replica (multi-process) path on CPU: world size 2 over gloo, no GPU.

Each rank owns a shard of the ensemble; lambda_TGF gathered over the ranks must equal the
single-process value, shards must partition the ensemble, and the timing max is a max.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, E, Q, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2107_03747_gb300 import replicas

        idx = replicas.shard(len(E), rank, world)
        lam, kept = replicas.ensemble_lambda(0.3, 12, 0.18, [E[i] for i in idx], [Q[i] for i in idx])
        tmax = replicas.max_over_ranks(float(rank + 1))
        allidx = replicas.gather_values([float(i) for i in idx])
        out[rank] = (lam, kept, tmax, list(allidx))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def built():
    from paper_2107_03747_gb300 import build

    build.build()


def test_shard_partitions_the_ensemble():
    from paper_2107_03747_gb300 import replicas

    for n, w in [(16, 2), (256, 8), (7, 3), (3, 4)]:
        parts = [replicas.shard(n, r, w) for r in range(w)]
        flat = [i for p in parts for i in p]
        assert flat == list(range(n))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_two_rank_gloo_ensemble_lambda_matches_single_process(built):
    from oracle import tgf_oracle as O

    rng = np.random.default_rng(3)
    E = list(rng.uniform(0.05, 0.2, size=9))
    Q = list(rng.normal(0.0, 0.6, size=9))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, E, Q, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    lam_ref, kept_ref = O.lambda_tgf(0.3, 12, 0.18, E, Q)
    for r in range(2):
        lam, kept, tmax, allidx = res[r]
        assert kept == kept_ref
        assert lam == pytest.approx(lam_ref, rel=1e-12)
        assert tmax == 2.0
        assert allidx == [float(i) for i in range(9)]

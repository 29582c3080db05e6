"""Replica parallelism over configurations (one process per GPU).

Configurations of an ensemble are independent, so N processes each flow their own shard with
no exchange on the data path.  The only exchange is after the flow: lambda_TGF (eq.
lambdat_latt) is an ensemble average, so every rank contributes its configurations' (E, Q) at
the end time and the values are gathered on the host side of the process group (gloo or nccl).
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, rank: int, world: int):
    """Indices of the configurations owned by `rank`: a contiguous block, sizes differing by at most one."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))


def _device_for(group=None):
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    if backend == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_values(local, group=None) -> np.ndarray:
    """All-gather a variable-length 1-D float64 array from every rank, concatenated in rank order."""
    import torch
    import torch.distributed as dist

    dev = _device_for(group)
    world = dist.get_world_size(group)
    x = torch.as_tensor(np.asarray(local, dtype=np.float64), device=dev).reshape(-1)
    n = torch.tensor([x.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(int(s.item()) for s in sizes))
    pad = torch.zeros(m, dtype=torch.float64, device=dev)
    pad[: x.numel()] = x
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return np.concatenate([p[: int(s.item())].cpu().numpy() for p, s in zip(parts, sizes)])


def max_over_ranks(x: float, group=None) -> float:
    """The maximum of a scalar over the ranks (the timing rule of the benchmark)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=_device_for(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def ensemble_lambda(c: float, Lt: int, t: float, E_local, Q_local, group=None):
    """lambda_TGF over the configurations of all ranks: (lambda or None, number kept)."""
    from paper_2107_03747_gb300 import binding

    E = gather_values(E_local, group)
    Q = gather_values(Q_local, group)
    return binding.tgf_lambda(c, Lt, t, E, Q)

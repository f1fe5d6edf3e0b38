"""Sharding of independent (frequency, shot) solves across ranks, one GPU per rank.

Every (shot, frequency) solve of the misfit of Eq. 4 is independent, so a
multi-GPU run splits the pairs across ranks with no exchange on the data path;
the only collectives are one sum of the misfit and gradient at the end of a
gradient evaluation (the implicit sums over shots and frequencies of Eq. 4 and
Eq. 7) and, for timing, a max over ranks. The collectives go through
torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def shard_pairs(omegas, nshot: int, world: int, rank: int):
    """The (frequency index, shot index) pairs of this rank.

    Pairs are dealt greedily, most expensive first, to the least loaded rank;
    the expected cost of a solve grows with its frequency (iteration counts grow
    roughly linearly with omega). Deterministic for given inputs.
    """
    om = np.asarray(omegas, float).reshape(-1)
    pairs = [(f, s) for f in range(om.size) for s in range(nshot)]
    order = sorted(range(len(pairs)), key=lambda k: (-om[pairs[k][0]], k))
    load = np.zeros(world)
    mine = []
    for k in order:
        r = int(np.argmin(load))
        load[r] += om[pairs[k][0]]
        if r == rank:
            mine.append(pairs[k])
    return sorted(mine)


def group_by_frequency(pairs):
    """{frequency index: [shot indices]} for a rank's pairs (one batched call per frequency)."""
    out: dict[int, list[int]] = {}
    for f, s in pairs:
        out.setdefault(f, []).append(s)
    return out


def allreduce_sum(J: float, grad: np.ndarray):
    """Sum J and the gradient over all ranks (no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return J, grad
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.from_numpy(np.concatenate([[J], np.asarray(grad, np.float64).ravel()])).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    t = t.cpu().numpy()
    return float(t[0]), t[1:].reshape(np.shape(grad))


def allreduce_max(x: float) -> float:
    """Max of a scalar over ranks (the timed region's length)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

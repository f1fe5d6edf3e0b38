"""Multi-rank path on CPU: (frequency, shot) sharding and the end-of-gradient sum,
with world_size 2 over gloo. Each rank evaluates its share with the oracle (the
per-rank GPU gradient in a real run); the summed result must equal the
single-rank gradient."""
import os
import socket

import numpy as np
import pytest

from paper_1712_08743_gb300 import shard


def test_shard_pairs_cover_every_pair_once():
    om = 2 * np.pi * np.array([3.0, 4.0, 5.0, 6.0])
    for world in (1, 2, 3, 8):
        got = [p for r in range(world) for p in shard.shard_pairs(om, 32, world, r)]
        assert sorted(got) == [(f, s) for f in range(4) for s in range(32)]
        loads = [sum(om[f] for f, _ in shard.shard_pairs(om, 32, world, r)) for r in range(world)]
        assert max(loads) - min(loads) <= om.max() + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    import oracle
    from synth import models

    rng = np.random.default_rng(21)
    Px, Pz, h, npml = 30, 20, 10.0, 6
    c_true = models.layered_model(rng, Px, Pz, h, 3)
    c0 = np.full_like(c_true, c_true.mean())
    src = np.array([[4, 1], [12, 1], [20, 1], [27, 1]])
    rec = np.array([[i, 1] for i in range(0, Px, 3)])
    om = 2 * np.pi * np.array([7.0, 11.0])
    d_obs = np.stack([oracle.sample_receivers(oracle.solve_fields(1 / c_true, h, w, src, npml), rec, npml) for w in om])
    return 1 / c0, h, npml, src, rec, om, d_obs


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    m0, h, npml, src, rec, om, d_obs = _problem()
    J, g = 0.0, np.zeros_like(m0)
    for f, shots in shard.group_by_frequency(shard.shard_pairs(om, len(src), world, rank)).items():
        Jf, gf = oracle.gradient(m0, h, om[f:f + 1], src[shots], rec, d_obs[f:f + 1, shots], 0.0, npml)
        J += Jf
        g += gf
    J, g = shard.allreduce_sum(J, g)
    tmax = shard.allreduce_max(float(rank + 1))
    dist.destroy_process_group()
    q.put((rank, J, g, tmax))


@pytest.mark.timeout(300)
def test_two_rank_gradient_sum_equals_single_rank():
    import torch.multiprocessing as mp

    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m0, h, npml, src, rec, om, d_obs = _problem()
    lam = 1e-3
    Jr, gr = oracle.gradient(m0, h, om, src, rec, d_obs, lam, npml)
    for rank, J, g, tmax in out:
        # the regulariser is added once, after the sum
        assert abs(J + lam * np.sum(m0 ** 2) - Jr) / Jr < 1e-10
        assert np.linalg.norm(g + 2 * lam * m0 - gr) / np.linalg.norm(gr) < 1e-10
        assert tmax == 2.0

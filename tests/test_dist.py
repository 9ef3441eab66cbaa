"""Multi-rank host logic on CPU: two gloo ranks reproduce the single-rank results
of the HMF partial-sum exchange and of the Ring / 2D row split (the paper's
two-GPU scheme), with the oracle standing in for the per-rank compute."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1212_0262_gb300 import dist as D
from paper_1212_0262_gb300 import inputs


def test_shard_range_covers_everything_once():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [D.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def test_lpt_assignment_balances_ensemble_costs():
    n = inputs.ensemble_sizes(256, 1000).astype(np.float64)
    cost = n * n
    for world in (2, 4, 8):
        owner = D.lpt_assign(cost, world)
        loads = np.bincount(owner, weights=cost, minlength=world)
        # LPT: the busiest rank exceeds the mean by at most the largest item
        assert loads.max() - cost.sum() / world <= cost.max()
        assert np.array_equal(owner, D.lpt_assign(cost, world))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle as ora

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        # HMF: partial sums over the shard, exchanged, give the global magnetization
        N = 1001
        q, _ = inputs.waterbag(N, 3)
        lo, hi = D.shard_range(N, rank, world)
        part = np.array([np.cos(q[lo:hi]).sum(), np.sin(q[lo:hi]).sum()])
        res["hmf"] = D.allreduce_sums(part)
        # Ring / 2D: own rows of the force from all positions gathered from the shards
        for model, eps, n in ((1, 0.01, 77), (2, 1e-3, 64)):
            qq, _ = inputs.default_state(model, n, 5)
            d = 2 if model == 2 else 1
            lo, hi = D.shard_range(n, rank, world)
            comps = [D.allgather_shards(qq[c * n + lo:c * n + hi], n) for c in range(d)]
            full = np.concatenate(comps)
            f = ora.force_rows(model, full, np.arange(lo, hi), eps)
            res[f"force{model}"] = np.concatenate([D.allgather_shards(f[c], n) for c in range(d)])
        res["tmax"] = D.max_over_ranks(float(rank) + 0.5)
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_exchange_matches_single_rank():
    import oracle as ora

    ora.build()
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    q, _ = inputs.waterbag(1001, 3)
    for r in range(world):
        got = res[r]
        assert np.allclose(got["hmf"], [np.cos(q).sum(), np.sin(q).sum()], rtol=1e-14, atol=1e-12)
        assert np.array_equal(got["hmf"], res[0]["hmf"])  # same bits on every rank
        for model, eps, n in ((1, 0.01, 77), (2, 1e-3, 64)):
            qq, _ = inputs.default_state(model, n, 5)
            assert np.array_equal(got[f"force{model}"], ora.force(model, qq, eps))
        assert got["tmax"] == world - 0.5

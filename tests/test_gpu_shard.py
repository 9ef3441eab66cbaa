"""Row shards (md_shard_*): one system split among P = 2 and 4 contexts on one GPU,
exchanging their segments with cudaMemcpyAsync on separate streams after every
stage (the paper's two-GPU schemes, Sec. 3.1 last paragraph and Sec. 3.2 Fig. 2,
generalised to P ranks).

Compared with the FP64 oracle element by element (forces within 1e-12 / 2e-5 of
sum_j |f_ij|, states after 1 step within 1e-12 and after 10 steps within 1e-11 in
FP64) and with the same system advanced whole by md_step (the one-sided kernel:
every ordered pair, as the shards evaluate them): only the stream-K split of each
row's FP64 sum (Ring / 2D) or the order of the partial magnetizations (HMF)
differs, so agreement is to rounding."""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import MDError, ShardGroup, System, binding as B, inputs

pytestmark = pytest.mark.gpu

EPS = {0: 0.0, 1: 0.01, 2: 1e-3}
DT = {0: 0.1, 1: 0.05, 2: 0.01}
NS = {0: 4099, 1: 4097, 2: 4097}


def _whole(model, N, prec, seed=7):
    s = System(model, N, EPS[model], DT[model], seed, precision=prec)
    if model:
        s.set_tuning("symmetric", 0)  # every ordered pair, as the shards
    return s


@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_shard_initial_state_is_the_whole_systems_rows(model, P):
    N = NS[model]
    with ShardGroup(model, N, EPS[model], DT[model], 11, P) as g, System(model, N, EPS[model], DT[model], 11) as s:
        qg, pg = g.get_state()
        qs, ps = s.get_state()
        assert np.array_equal(qg, qs) and np.array_equal(pg, ps)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_shard_forces_match_the_oracle(model, P, prec):
    N = NS[model]
    q, p = inputs.default_state(model, N, 1000 + N)
    with ShardGroup(model, N, EPS[model], DT[model], 1, P, precision=prec) as g:
        g.set_state(q, p)
        f = g.force()
    fo = ora.force(model, q, EPS[model])
    scale = ora.force_abs(model, q, EPS[model])
    tol = 1e-12 if prec == "fp64" else 2e-5
    err = np.abs(f - fo)
    assert np.all(err <= tol * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()


@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_shard_steps_match_the_oracle_and_the_whole_system(model, P):
    N, dt = NS[model], DT[model]
    q0, p0 = inputs.default_state(model, N, 1000 + N)
    fs = ora.force_abs(model, q0, EPS[model]).max()
    with ShardGroup(model, N, EPS[model], dt, 1, P) as g, _whole(model, N, "fp64") as s:
        g.set_state(q0, p0)
        s.set_state(q0, p0)
        g.step(1)
        s.step(1)
        q, p = g.get_state()
        qo, po = ora.step(model, q0, p0, EPS[model], dt, 1)
        assert np.max(np.abs(q - qo)) <= 1e-12 * max(1.0, np.abs(qo).max())
        assert np.max(np.abs(p - po)) <= 1e-12 * (np.abs(po).max() + dt * fs)
        qs, ps = s.get_state()
        assert np.max(np.abs(q - qs)) <= 1e-12 * max(1.0, np.abs(qs).max())
        assert np.max(np.abs(p - ps)) <= 1e-12 * (np.abs(ps).max() + dt * fs)
        g.step(4)
        g.step(5)  # two calls: every call closes with a kick and restarts from the exchanged state
        s.step(9)
        q, p = g.get_state()
        qo, po = ora.step(model, q0, p0, EPS[model], dt, 10)
        assert np.max(np.abs(q - qo)) <= 1e-11 * max(1.0, np.abs(qo).max())
        assert np.max(np.abs(p - po)) <= 1e-11 * max(1.0, np.abs(po).max())
        qs, ps = s.get_state()
        assert np.max(np.abs(q - qs)) <= 1e-11 * max(1.0, np.abs(qs).max())
        assert np.max(np.abs(p - ps)) <= 1e-11 * max(1.0, np.abs(ps).max())


@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_mixed_shard_steps_match_the_whole_mixed_system(model, P):
    """Mixed precision: the same FP32 pair terms (or sines and cosines) on both sides.
    Ring / 2D: the FP64 sums of FP32 tile sums are grouped differently, so 1e-9 as for
    ensembles.  HMF: each thread adds its sines and cosines in FP32 before the FP64
    sum, and the shards group the N angles differently, so the magnetizations may
    differ by up to u32 = 2^-24 (N terms of magnitude <= 1, over N), the forces by
    2 u32, and after n steps p by n sum|b| dt 2 u32 and q by that times sum|d| dt n."""
    N, dt = NS[model], DT[model]
    nsteps = 10
    q0, p0 = inputs.default_state(model, N, 2000 + N)
    with ShardGroup(model, N, EPS[model], dt, 1, P, precision="mixed") as g, _whole(model, N, "mixed") as s:
        g.set_state(q0, p0)
        s.set_state(q0, p0)
        g.step(nsteps)
        s.step(nsteps)
        q, p = g.get_state()
        qs, ps = s.get_state()
    if model == 0:
        B0, B1, D0, D1 = ora.yoshida()
        bp = nsteps * (2 * abs(B0) + 2 * abs(B1)) * dt * 2 * 2.0 ** -24
        bq = bp * (2 * abs(D0) + abs(D1)) * dt * nsteps
    else:
        bq, bp = 1e-9 * max(1.0, np.abs(qs).max()), 1e-9 * max(1.0, np.abs(ps).max())
    assert np.max(np.abs(q - qs)) <= bq, (np.max(np.abs(q - qs)), bq)
    assert np.max(np.abs(p - ps)) <= bp, (np.max(np.abs(p - ps)), bp)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_shard_runs_are_bitwise_deterministic(model, prec):
    out = []
    for _ in range(2):
        with ShardGroup(model, NS[model], EPS[model], DT[model], 5, 3, precision=prec) as g:
            g.step(6)
            out.append(g.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("model", [1, 2])
def test_benchmark_size_shard_forces_match_sampled_oracle_rows(model):
    """Ring N = 131,072 and 2D N = 262,144 (the benchmark sizes) split over 4 ranks,
    mixed precision: 64 sampled rows from every rank against ora.force_rows."""
    N = 131_072 if model == 1 else 262_144
    eps = 0.01 if model == 1 else 1e-4
    with ShardGroup(model, N, eps, DT[model], 3 if model == 1 else 4, 4, precision="mixed") as g:
        q, _ = g.get_state()
        g.begin()
        f = g.force().reshape(-1, N)
        rng = np.random.default_rng(9)
        rows = np.unique(np.concatenate([rng.integers(lo, hi, 16) for lo, hi in g.ranges] +
                                        [[lo, hi - 1] for lo, hi in g.ranges]))
    fo, scale = ora.force_rows(model, q, rows, eps, with_abs=True)
    err = np.abs(f[:, rows] - fo)
    assert np.all(err <= 2e-5 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()


class _DeviceBytes:
    """A view of n device bytes for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False), "version": 3}


@pytest.mark.parametrize("model", [0, 1, 2])
def test_exchange_buffers_hold_every_ranks_segment(model):
    """After md_shard_begin and the exchange, every rank's buffer holds the same bytes:
    each segment written by its owner and copied into the others; segments tile the
    buffer in rank order."""
    import torch

    with ShardGroup(model, NS[model], EPS[model], DT[model], 3, 4, precision="mixed") as g:
        g.begin()
        for _ in range(2):
            g.synchronize()
            segs = [g.buffer(r) for r in range(4)]
            total = segs[-1][1] + segs[-1][2]
            assert segs[0][1] == 0
            assert all(segs[r][1] + segs[r][2] == segs[r + 1][1] for r in range(3))
            host = [torch.as_tensor(_DeviceBytes(ptr, total), device="cuda").cpu().numpy() for ptr, _, _ in segs]
            for h in host[1:]:
                assert np.array_equal(h, host[0])
            g.stage(0.6, 1.3)  # and again after a stage (the other buffer of the pair)


def test_shard_misuse_is_reported():
    with ShardGroup(1, 4097, 0.01, 0.05, 1, 2) as g:
        lib = B.load()
        assert lib.md_shard_stage(g._h(0), 1.0, 1.0) == B.MD_ESTATE  # before md_shard_begin
        assert lib.md_step(g._h(0), 1) == B.MD_ESTATE
        assert lib.md_energy(g._h(0), None, None) == B.MD_ESTATE
        g.begin()
        swapped = (type(g._ctx)._type_ * 2)(g._ctx[1], g._ctx[0])
        assert lib.md_shard_exchange(swapped, 2) == B.MD_EINVAL
        g.set_precision("mixed")
        with pytest.raises(MDError) as e:
            g.stage(1.0, 1.0)  # precision changed since md_shard_begin
        assert e.value.code == B.MD_ESTATE
        g.step(1)  # md_shard_step begins again by itself
    with pytest.raises(MDError) as e:
        ShardGroup(2, 2000, 1e-3, 0.01, 1, 4)
    assert e.value.code == B.MD_EINVAL

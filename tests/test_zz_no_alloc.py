"""md_potential_noalloc: the potential energy for callers that cannot allocate
device memory (their GPU memory belongs to a host framework's caching
allocator, or cudaMalloc's possible device synchronisation is not acceptable in
their loop).  Its scratch is a static device array, so two calls in a row must
both agree with md_energy's V, the entry point that allocates its scratch, and with
the FP64 oracle's i<j pair sum (1e-12 relative).

This file is collected last on purpose; it needs nothing from the other tests.
"""
import ctypes
import functools

import numpy as np
import pytest
import torch

import oracle as ora
from paper_1212_0262_gb300 import System, binding, inputs


@functools.lru_cache(maxsize=None)
def _oracle_potential(model, N, eps, seed):
    q, _ = inputs.default_state(model, N, seed)
    return ora.potential(model, q, eps)


def _oracle_tol(model, N):
    """Relative tolerance against the oracle: 1e-12, or the oracle's own rounding
    where it is larger.  The oracle adds the N (N - 1) / 2 pair terms one by one in
    FP64, so its sum carries a rounding error of order sqrt(n) u relative (u = 2^-53;
    n u in the worst case): about 5e-12 for the 2.1e9 pairs at N = 65536."""
    n = N if model == 0 else N * (N - 1) / 2
    return max(1e-12, 4.0 * np.sqrt(n) * 2.0 ** -53)

pytestmark = pytest.mark.gpu

CASES = [(0, 65536, 0.0), (1, 4097, 0.01), (2, 65536, 1e-4), (1, 1, 0.01), (2, 333, 1e-3), (3, 65536, 1e-3),
         (3, 1, 1e-3), (4, 65536, 0.0), (4, 777, 1e-3)]


def _noalloc(model, N, eps, q_dev, v_dev, stream):
    lib = binding.load()
    return lib.md_potential_noalloc(model, N, eps, ctypes.c_void_p(q_dev.data_ptr()),
                                    ctypes.c_void_p(v_dev.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("model,N,eps", CASES)
def test_noalloc_potential_matches_md_energy_twice(model, N, eps):
    q, p = inputs.default_state(model, N, 500 + N)
    with System(model, N, eps, 0.01, 1) as s:
        s.set_state(q, p)
        _, v_ref = s.energy()
    q_dev = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    v_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        v_dev.fill_(float("nan"))
        rc = _noalloc(model, N, eps, q_dev, v_dev, stream)
        assert rc == 0, binding.load().md_last_error(None)
        torch.cuda.synchronize()
        v = float(v_dev.item())
        assert abs(v - v_ref) <= 1e-12 * max(abs(v_ref), 1.0), (call, v, v_ref)
    v_ora = _oracle_potential(model, N, eps, 500 + N)
    assert abs(v - v_ora) <= _oracle_tol(model, N) * max(abs(v_ora), 1.0), (v, v_ora)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    q_dev = torch.zeros(65537, dtype=torch.float64, device="cuda")
    v_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = _noalloc(1, 65537, 0.01, q_dev, v_dev, torch.cuda.current_stream())
    assert rc == binding.MD_EINVAL
    assert b"65536" in binding.load().md_last_error(None)


def test_noalloc_alternating_models_keep_agreeing():
    """The shared array keeps the previous call's contents; a call of another
    model and size in between must not change the answer."""
    stream = torch.cuda.current_stream()
    qa, pa = inputs.default_state(2, 1000, 3)
    qb, pb = inputs.default_state(1, 70, 4)
    with System(2, 1000, 1e-3, 0.01, 1) as s:
        s.set_state(qa, pa)
        _, va = s.energy()
    qa_dev = torch.from_numpy(qa).cuda()
    qb_dev = torch.from_numpy(qb).cuda()
    v_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _noalloc(2, 1000, 1e-3, qa_dev, v_dev, stream) == 0
        torch.cuda.synchronize()
        assert abs(v_dev.item() - va) <= 1e-12 * abs(va)
        assert _noalloc(1, 70, 0.01, qb_dev, v_dev, stream) == 0
        torch.cuda.synchronize()


def test_noalloc_calls_on_two_streams_and_threads_do_not_race():
    """Calls queued on two streams without any synchronisation between them, and from
    two host threads, share the static scratch: each waits on the GPU for the previous
    call, so every value equals md_energy's."""
    import threading

    cases = [(2, 65536, 1e-4, 11), (1, 4097, 0.01, 12)]
    refs, qs = [], []
    for model, N, eps, seed in cases:
        q, p = inputs.default_state(model, N, seed)
        with System(model, N, eps, 0.01, 1) as s:
            s.set_state(q, p)
            refs.append(s.energy()[1])
        qs.append(torch.from_numpy(np.ascontiguousarray(q)).cuda())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out = torch.full((2, 16), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for k in range(16):
        for c, (model, N, eps, _) in enumerate(cases):
            assert _noalloc(model, N, eps, qs[c], out[c, k:k + 1], streams[c]) == 0
    torch.cuda.synchronize()
    for c in range(2):
        v = out[c].cpu().numpy()
        assert np.all(np.abs(v - refs[c]) <= 1e-12 * abs(refs[c])), (c, v, refs[c])

    out.fill_(float("nan"))
    torch.cuda.synchronize()
    errors = []

    def worker(c):
        model, N, eps, _ = cases[c]
        try:
            for k in range(16):
                rc = _noalloc(model, N, eps, qs[c], out[c, k:k + 1], streams[c])
                if rc:
                    errors.append((c, rc))
        except Exception as e:  # reported below
            errors.append((c, repr(e)))

    ts = [threading.Thread(target=worker, args=(c,)) for c in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=120)
    torch.cuda.synchronize()
    assert not errors, errors
    for c in range(2):
        v = out[c].cpu().numpy()
        assert np.all(np.abs(v - refs[c]) <= 1e-12 * abs(refs[c])), (c, v, refs[c])


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("model", [1, 2, 3])
def test_noalloc_potential_of_a_non_finite_position_is_not_finite(model, bad):
    """A NaN or infinite coordinate gives a V that is not finite (never a finite number
    that looks valid), and the next call on a good state is right again."""
    N, eps = 1000, {1: 0.01, 2: 1e-3, 3: 1e-3}[model]
    q, _ = inputs.default_state(model, N, 21)
    qb = q.copy()
    qb[333] = bad
    stream = torch.cuda.current_stream()
    v_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(model, N, eps, torch.from_numpy(qb).cuda(), v_dev, stream) == 0
    torch.cuda.synchronize()
    assert not np.isfinite(v_dev.item())
    assert _noalloc(model, N, eps, torch.from_numpy(q).cuda(), v_dev, stream) == 0
    torch.cuda.synchronize()
    v_ora = _oracle_potential(model, N, eps, 21)
    assert abs(v_dev.item() - v_ora) <= 1e-12 * max(abs(v_ora), 1.0)

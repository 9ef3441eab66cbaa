"""Host logic of the row shards (md_shard_range and argument checks): no GPU needed.

The split generalises the paper's two-GPU schemes (Sec. 3.1 last paragraph, Sec. 3.2
Fig. 2) to P ranks: contiguous row ranges covering [0, N) in rank order, starting on
whole 1024-row blocks for Ring and 2D (whole mirror record groups and i-tiles), on
any row for HMF, and no empty rank."""
import ctypes

import pytest

from paper_1212_0262_gb300 import binding as B


@pytest.fixture(scope="module")
def lib():
    from paper_1212_0262_gb300 import build

    build.build()
    return B.load()


def _range(lib, model, N, r, P):
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.md_shard_range(model, N, r, P, ctypes.byref(lo), ctypes.byref(hi))
    return rc, lo.value, hi.value


@pytest.mark.parametrize("model,N,P", [(0, 4099, 4), (0, 5, 5), (0, 50_000_000, 8), (1, 4097, 4), (2, 262_144, 4),
                                       (2, 1_000_003, 8), (1, 2048, 2), (0, 1, 1), (2, 7, 1), (1, 131_072, 64)])
def test_ranges_tile_the_rows_in_rank_order(lib, model, N, P):
    bounds = []
    for r in range(P):
        rc, lo, hi = _range(lib, model, N, r, P)
        assert rc == 0
        assert hi > lo
        if model != 0:
            assert lo % 1024 == 0
        bounds.append((lo, hi))
    assert bounds[0][0] == 0 and bounds[-1][1] == N
    assert all(bounds[r][1] == bounds[r + 1][0] for r in range(P - 1))
    # near-even split: no rank holds more than its share plus one block
    share = N / P
    assert max(hi - lo for lo, hi in bounds) <= share + (1 if model == 0 else 1024) + 1


@pytest.mark.parametrize("model,N,P", [(1, 2000, 4), (2, 1023, 2), (0, 3, 4), (1, 4096, 65), (3, 4096, 2),
                                       (4, 4096, 2), (1, 0, 1)])
def test_impossible_splits_are_rejected(lib, model, N, P):
    rc, _, _ = _range(lib, model, N, 0, P)
    assert rc == B.MD_EINVAL
    assert lib.md_last_error(None)


def test_shard_calls_reject_missing_or_whole_system_contexts(lib):
    assert lib.md_shard_begin(None) == B.MD_EINVAL
    assert lib.md_shard_stage(None, 1.0, 1.0) == B.MD_EINVAL
    assert lib.md_shard_force(None, None) == B.MD_EINVAL
    assert lib.md_shard_exchange(None, 2) == B.MD_EINVAL
    assert lib.md_shard_step(None, 0, 1) == B.MD_EINVAL
    rc, _, _ = _range(lib, 1, 4097, 4, 4)  # rank out of range
    assert rc == B.MD_EINVAL

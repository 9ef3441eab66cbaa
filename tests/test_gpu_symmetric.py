"""Newton's-third-law variant of the FP32 Ring and 2D stages against the FP64
oracle, through the C ABI (needs a GB300).

Every unordered pair is evaluated once; the term enters particle i's sum through
the row partial and particle j's (negated) through a per-unit column partial.
Tolerances are those of the one-sided FP32 kernels: |f - f_ora| <= 2e-5 sum_j |f_ij|.
Sizes span one to many i-tiles (Ring: 256 particles, 2D: 1024) with ragged tails.
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs

pytestmark = pytest.mark.gpu

EPS = {1: 0.01, 2: 1e-3}
SIZES = [1, 2, 3, 33, 255, 256, 257, 1000, 1024, 1025, 2049, 4097, 9000]


KERNEL = {(1, 1): 5, (2, 1): 4, (1, 0): 3, (2, 0): 2}  # MD_KERNEL_* by (model, symmetric)


def _sym(model, N, dt=0.05, seed=7, symmetric=1):
    s = System(model, N, EPS[model], dt, seed, precision="mixed")
    if model == 1:
        s.set_tuning("ring_tc", 1)
    s.set_tuning("symmetric", symmetric)
    assert s.force_kernel == KERNEL[(model, symmetric)]
    q, p = inputs.default_state(model, N, 1000 + N)
    s.set_state(q, p)
    return s, q, p


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("model", [1, 2])
def test_symmetric_force_error_bound(model, N):
    s, q, _ = _sym(model, N)
    f = s.force()
    fo = ora.force(model, q, EPS[model])
    scale = ora.force_abs(model, q, EPS[model])
    err = np.abs(f - fo)
    assert np.all(err <= 2e-5 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()
    if N == 1:
        assert np.all(f == 0.0)


@pytest.mark.parametrize("model", [1, 2])
def test_symmetric_force_differs_from_one_sided_only_by_rounding(model):
    """Both kernels evaluate the same pair terms; only the summation order differs."""
    N = 5000
    s, q, _ = _sym(model, N)
    o, _, _ = _sym(model, N, symmetric=0)
    f, g = s.force(), o.force()
    scale = ora.force_abs(model, q, EPS[model])
    assert not np.array_equal(f, g)  # the two kernels did run
    assert np.all(np.abs(f - g) <= 2e-5 * scale)


@pytest.mark.parametrize("model", [1, 2])
def test_symmetric_steps_track_fp64(model):
    """Ten steps (kick-drift, kick-only and first-same-as-last stages) stay as
    close to the FP64 path as the one-sided FP32 kernel does, and the energy error
    keeps the mixed-vs-FP64 bound."""
    N, dt = 3000, (0.05 if model == 1 else 0.01)
    ref = System(model, N, EPS[model], dt, 7, precision="fp64")
    q0, p0 = inputs.default_state(model, N, 1000 + N)
    ref.set_state(q0, p0)
    s, _, _ = _sym(model, N, dt=dt)
    o, _, _ = _sym(model, N, dt=dt, symmetric=0)
    e0 = sum(ref.energy())
    for x in (ref, s, o):
        x.step(4)
        x.step(6)
    (qr, pr), (qs, ps), (qo, po) = ref.get_state(), s.get_state(), o.get_state()
    d_sym = max(np.abs(qs - qr).max(), np.abs(ps - pr).max())
    d_one = max(np.abs(qo - qr).max(), np.abs(po - pr).max())
    assert d_sym < 1e-5 and d_sym <= 4 * d_one + 1e-9, (d_sym, d_one)
    de_ref = abs(sum(ref.energy()) - e0) / abs(e0)
    de_sym = abs(sum(s.energy()) - e0) / abs(e0)
    assert de_sym <= 2 * de_ref + 1e-9, (de_sym, de_ref)


@pytest.mark.parametrize("model", [1, 2])
def test_symmetric_runs_are_bitwise_deterministic(model):
    out = []
    for _ in range(2):
        s, _, _ = _sym(model, 6000)
        s.step(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("model", [1, 2])
def test_symmetric_total_momentum_conserved(model):
    N = 4097
    s, q0, p0 = _sym(model, N)
    s.step(20)
    q, p = s.get_state()
    d = 2 if model == 2 else 1
    for c in range(d):
        drift = abs(p[c * N:(c + 1) * N].sum() - p0[c * N:(c + 1) * N].sum())
        assert drift < 1e-6 * np.abs(p0).sum(), drift


@pytest.mark.parametrize("model,N,eps", [(1, 131072, 0.01), (2, 262144, 1e-4)])
def test_symmetric_full_size_sampled_force_parity(model, N, eps):
    """Bench-size systems in the bench's launch configuration: forces on 64
    sampled particles against the oracle's direct sums."""
    s = System(model, N, eps, 0.05, 42 + model, precision="mixed")
    if model == 1:
        s.set_tuning("ring_tc", 1)
    s.set_tuning("symmetric", 1)
    assert s.force_kernel == KERNEL[(model, 1)]
    q, _ = s.get_state()
    f = s.force().reshape(2 if model == 2 else 1, N)
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(9, np.arange(62)) % np.uint64(N)]).astype(np.int64))
    fo, scale = ora.force_rows(model, q, rows, eps, with_abs=True)
    assert np.all(np.abs(f[:, rows] - fo) <= 2e-5 * scale), (np.abs(f[:, rows] - fo) / scale).max()
    s.close()


def test_symmetric_falls_back_to_one_sided_beyond_the_column_cap():
    """Ring N = 1,572,864 needs 19.3 GB of column partials, beyond the 16 GiB cap: the
    one-sided tensor-core kernel runs instead, with the same error bound."""
    N = 3 << 19
    s = System(1, N, 0.01, 0.05, 47, precision="mixed")
    assert s.force_kernel == 3  # one-sided, tensor-core products
    q, _ = s.get_state()
    f = s.force()
    rows = np.array([0, 12345, N - 1])
    fo, scale = ora.force_rows(1, q, rows, 0.01, with_abs=True)
    assert np.all(np.abs(f[rows] - fo[0]) <= 2e-5 * scale[0])
    s.close()


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("model", [1, 2])
def test_stream_k_range_counts_keep_parity(model, symmetric):
    """pair_vcta: the units split into 1, 3, 5 or 32 ranges per resident CTA (fewer
    where that would leave under 16 units a range), taken by the CTAs from a counter
    that the launch's last CTA sets back to 0.  Forces match the oracle within the
    FP32 bound for every split, over several consecutive launches (a counter left
    non-zero would skip ranges of the next launch), and a split gives the same bits
    every time."""
    N = 40_000
    q, _ = inputs.default_state(model, N, 1000 + N)
    fo = ora.force(model, q, EPS[model])
    scale = ora.force_abs(model, q, EPS[model])
    for k in (1, 3, 5, 32):
        s, _, _ = _sym(model, N, symmetric=symmetric)
        s.set_tuning("pair_vcta", k)
        s.set_state(q, np.zeros_like(q))
        fs = [s.force() for _ in range(3)]
        for f in fs:
            err = np.abs(f - fo)
            assert np.all(err <= 2e-5 * scale + 1e-300), (k, (err / np.maximum(scale, 1e-300)).max())
        assert np.array_equal(fs[0], fs[1]) and np.array_equal(fs[0], fs[2]), k
        s.close()

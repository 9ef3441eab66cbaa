"""2D FP32 stages with the coordinate differences on the tensor cores (tuning key
grav_tc), against the FP64 oracle through the C ABI (needs a GB300).

dx = x_i - x_j and dy come from one m16n8k8 TF32 product each, with every FP32
coordinate split exactly into three TF32 parts; the rest of the pair arithmetic
is the FP32 kernel's.  Tolerance: that of the FP32 kernels,
|f - f_ora| <= 2e-5 sum_j |f_ij|.  Sizes span one to many 256-particle tiles with
ragged tails; the three symmetric CTA shapes and the one-sided kernel.
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-3
SIZES = [1, 2, 3, 33, 255, 256, 257, 1000, 1025, 4097, 9000]
KERNEL = {1: 5, 0: 3}  # MD_KERNEL_PAIRS_TC_SYM / MD_KERNEL_PAIRS_TC by symmetric


def _sys(N, variant=1, symmetric=1, dt=0.01, seed=7, eps=EPS):
    s = System(2, N, eps, dt, seed, precision="mixed")
    s.set_tuning("grav_tc", variant)
    s.set_tuning("symmetric", symmetric)
    q, p = inputs.default_state(2, N, 1000 + N)
    s.set_state(q, p)
    return s, q, p


def _check(f, q, eps=EPS):
    fo = ora.force(2, q, eps)
    scale = ora.force_abs(2, q, eps)
    err = np.abs(f - fo)
    assert np.all(err <= 2e-5 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_symmetric_tc_force_error_bound(variant, N):
    s, q, _ = _sys(N, variant)
    if N >= 2:
        assert s.force_kernel == KERNEL[1]
    f = s.force()
    _check(f, q)
    if N == 1:
        assert np.all(f == 0.0)


@pytest.mark.parametrize("N", SIZES)
def test_one_sided_tc_force_error_bound(N):
    s, q, _ = _sys(N, 1, symmetric=0)
    assert s.force_kernel == KERNEL[0]
    _check(s.force(), q)


def test_coincident_particles():
    """Duplicated positions off the diagonal: dx = dy = 0 exactly, a zero term."""
    N = 1000
    q, _ = inputs.default_state(2, N, 5)
    q = q.copy()
    for a, b in ((10, 11), (300, 700), (998, 999)):
        q[a], q[N + a] = q[b], q[N + b]
    s = System(2, N, EPS, 0.01, 1, precision="mixed")
    s.set_tuning("grav_tc", 1)
    s.set_state(q, np.zeros_like(q))
    _check(s.force(), q)


def test_far_coordinates_within_one_more_rounding():
    """Coordinates near (1e3, -1e3), where FP32 positions resolve only 6e-5: against
    the oracle on the FP32-rounded positions, the error stays within the FP32
    kernels' bound plus one more rounding of dx and dy at the coordinates' scale
    (the tensor core accumulates the six split parts in FP32):
    |df_i| <= 2e-5 sum_j |f_ij| + (2/N) sum_j 3 (2 ulp(|x|max)) / s_ij."""
    N = 1000
    q, _ = inputs.default_state(2, N, 5)
    q = q.copy()
    q[:N] += 1.0e3
    q[N:] -= 1.0e3
    q32 = q.astype(np.float32).astype(np.float64)
    s = System(2, N, EPS, 0.01, 1, precision="mixed")
    s.set_tuning("grav_tc", 1)
    s.set_state(q, np.zeros_like(q))
    f = s.force()
    fo = ora.force(2, q32, EPS)
    scale = ora.force_abs(2, q32, EPS)
    x, y = q32[:N], q32[N:]
    dx, dy = x[:, None] - x[None, :], y[:, None] - y[None, :]
    inv = 1.0 / (dx * dx + dy * dy + EPS)
    np.fill_diagonal(inv, 0.0)
    ulp = float(np.spacing(np.float32(np.abs(q32).max())))
    extra = (2.0 / N) * 3.0 * (2.0 * ulp) * inv.sum(axis=1)
    bound = 2e-5 * scale + np.concatenate([extra, extra])
    err = np.abs(f - fo)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("variant", [1, 2])
def test_tc_steps_track_fp64(variant):
    """Ten steps (kick-drift, kick-only and first-same-as-last stages) stay as close
    to the FP64 path as the plain FP32 kernel does; the energy error keeps the
    mixed-vs-FP64 bound."""
    N, dt = 3000, 0.01
    ref = System(2, N, EPS, dt, 7, precision="fp64")
    q0, p0 = inputs.default_state(2, N, 1000 + N)
    ref.set_state(q0, p0)
    s, _, _ = _sys(N, variant, dt=dt)
    o, _, _ = _sys(N, 0, dt=dt)
    e0 = sum(ref.energy())
    for x in (ref, s, o):
        x.step(4)
        x.step(6)
    (qr, pr), (qs, ps), (qo, po) = ref.get_state(), s.get_state(), o.get_state()
    d_tc = max(np.abs(qs - qr).max(), np.abs(ps - pr).max())
    d_cc = max(np.abs(qo - qr).max(), np.abs(po - pr).max())
    assert d_tc < 1e-5 and d_tc <= 4 * d_cc + 1e-9, (d_tc, d_cc)
    de_ref = abs(sum(ref.energy()) - e0) / abs(e0)
    de_tc = abs(sum(s.energy()) - e0) / abs(e0)
    assert de_tc <= 2 * de_ref + 1e-9, (de_tc, de_ref)


def test_tc_runs_are_bitwise_deterministic():
    out = []
    for _ in range(2):
        s, _, _ = _sys(6000, 1)
        s.step(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_switching_record_format_mid_run():
    """grav_tc on, off and on again between steps: each change rewrites the mirror
    in the other record format; the trajectory stays within the FP32 bound of an
    FP64 run."""
    N, dt = 2049, 0.01
    ref = System(2, N, EPS, dt, 7, precision="fp64")
    q0, p0 = inputs.default_state(2, N, 33)
    ref.set_state(q0, p0)
    s = System(2, N, EPS, dt, 7, precision="mixed")
    s.set_state(q0, p0)
    for v in (1, 0, 2, 0, 1):
        s.set_tuning("grav_tc", v)
        s.step(2)
    ref.step(10)
    (qr, pr), (qs, ps) = ref.get_state(), s.get_state()
    assert max(np.abs(qs - qr).max(), np.abs(ps - pr).max()) < 1e-5


def test_tc_full_size_sampled_force_parity():
    """The bench's 2D system (N = 262,144, eps = 1e-4) in the bench's launch
    configuration: forces on 64 sampled particles against the oracle's direct sums."""
    N, eps = 262144, 1e-4
    s = System(2, N, eps, 0.01, 44, precision="mixed")
    s.set_tuning("grav_tc", 1)
    assert s.force_kernel == KERNEL[1]
    q, _ = s.get_state()
    f = s.force().reshape(2, N)
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(9, np.arange(62)) % np.uint64(N)]).astype(np.int64))
    fo, scale = ora.force_rows(2, q, rows, eps, with_abs=True)
    assert np.all(np.abs(f[:, rows] - fo) <= 2e-5 * scale), (np.abs(f[:, rows] - fo) / scale).max()
    s.close()

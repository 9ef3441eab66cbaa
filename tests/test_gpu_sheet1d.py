"""1D self-gravitating sheets (MD_SHEET1D; named in the paper's introduction, not
one of its three models) through the C ABI against the FP64 oracle (needs a GB300).

eps = 0: f_i = -(1/N) sum_j sign(x_i - x_j) is an exact count divided by N, so the
FP64 path equals the oracle bit for bit, and the FP32 path (signs decided on the
FP32-rounded positions) equals the oracle's FP32-decision variant bit for bit.
eps > 0: d / sqrt(d^2 + eps) with the usual tolerances (1e-12 and 2e-5 of
sum_j |f_ij|).  Both kernel forms; sizes span one to many i-tiles with ragged tails.
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import MDError, System, inputs

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 33, 511, 1023, 1024, 1025, 2049, 4097]
KERNEL = {("fp64", 1): 6, ("fp64", 0): 1, ("mixed", 1): 4, ("mixed", 0): 2}


def _sys(N, prec="fp64", eps=0.0, symmetric=1, dt=0.01, seed=7):
    s = System(4, N, eps, dt, seed, precision=prec)
    s.set_tuning("symmetric", symmetric)
    assert s.force_kernel == KERNEL[(prec, symmetric)]
    q, p = inputs.sheet_state(N, 1000 + N)
    s.set_state(q, p)
    return s, q, p


def test_device_initial_state_matches_input_generator():
    with System(4, 5000, 0.0, 0.01, 1234) as s:
        q, p = s.get_state()
    qe, pe = inputs.sheet_state(5000, 1234)
    assert np.array_equal(q, qe) and np.array_equal(p, pe)


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("N", SIZES)
def test_exact_sign_force_fp64_bitwise(N, symmetric):
    s, q, _ = _sys(N, "fp64", 0.0, symmetric)
    f = s.force()
    assert np.array_equal(f, ora.force(4, q, 0.0))


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("N", SIZES)
def test_exact_sign_force_mixed_bitwise_with_fp32_decisions(N, symmetric):
    s, q, _ = _sys(N, "mixed", 0.0, symmetric)
    f = s.force()
    assert np.array_equal(f, ora.force_sheet_f32(q))


def test_mixed_fp32_ties_count_as_zero():
    """Two sheets that coincide in FP32 but not in FP64: the FP32 path takes the
    FP32 decision (sign 0), the FP64 path the FP64 one."""
    q = np.array([0.5, 0.5 + 1e-12, -0.25, 0.7])
    p = np.zeros(4)
    out = {}
    for prec in ("fp64", "mixed"):
        with System(4, 4, 0.0, 0.01, 1, precision=prec) as s:
            s.set_state(q, p)
            out[prec] = s.force()
    assert np.array_equal(out["fp64"], ora.force(4, q, 0.0))
    assert np.array_equal(out["mixed"], ora.force_sheet_f32(q))
    assert out["fp64"][0] != out["mixed"][0]


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
@pytest.mark.parametrize("N", [1, 33, 1025, 4097])
def test_softened_force_parity(N, prec, tol, symmetric):
    s, q, _ = _sys(N, prec, 1e-3, symmetric)
    f = s.force()
    err = np.abs(f - ora.force(4, q, 1e-3))
    scale = ora.force_abs(4, q, 1e-3)
    assert np.all(err <= tol * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_fp64_steps_parity(eps):
    dt = 0.01
    s, q0, p0 = _sys(33, eps=eps, dt=dt)
    s.step(4)
    s.step(6)
    q, p = s.get_state()
    qo, po = ora.step(4, q0, p0, eps, dt, 10)
    assert np.max(np.abs(q - qo)) <= 1e-11 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-11 * max(1.0, np.abs(po).max())


@pytest.mark.parametrize("eps", [0.0, 1e-3])
@pytest.mark.parametrize("N", [1, 2, 33, 1025, 4097])
def test_energy_parity(N, eps):
    s, q, p = _sys(N, eps=eps)
    K, V = s.energy()
    assert abs(K - ora.kinetic(p)) <= 1e-12 * max(abs(K), 1e-300)
    Vo = ora.potential(4, q, eps)
    assert abs(V - Vo) <= 1e-12 * max(abs(Vo), 1.0), (V, Vo)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_momentum_is_conserved_exactly_at_eps0(prec):
    """At eps = 0 the forces are exact multiples of 1/N that sum to zero, so the
    total momentum changes only by the rounding of the kicks."""
    N = 4097
    s, q0, p0 = _sys(N, prec)
    f = s.force()
    assert np.sum(f * N) == 0.0
    s.step(20)
    _, p = s.get_state()
    assert abs(p.sum() - p0.sum()) < 1e-12 * np.abs(p0).sum()


def test_eps_change_rewrites_the_padding():
    """Switching between the exact and the softened force changes the padding records
    (NaN for eps = 0, far away for eps > 0): forces stay right after md_set_eps."""
    s, q, _ = _sys(1000, "mixed", 0.0)
    assert np.array_equal(s.force(), ora.force_sheet_f32(q))
    s.set_eps(1e-3)
    err = np.abs(s.force() - ora.force(4, q, 1e-3))
    assert np.all(err <= 2e-5 * ora.force_abs(4, q, 1e-3))
    s.set_eps(0.0)
    assert np.array_equal(s.force(), ora.force_sheet_f32(q))


def test_runs_are_bitwise_deterministic():
    out = []
    for _ in range(2):
        s, _, _ = _sys(3000, "mixed", 1e-3)
        s.step(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_sampled_force_parity(prec):
    N = 262144
    s = System(4, N, 0.0, 0.01, 46, precision=prec)
    q, _ = s.get_state()
    f = s.force()
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(9, np.arange(62)) % np.uint64(N)]).astype(np.int64))
    if prec == "fp64":
        fo = ora.force_rows(4, q, rows, 0.0)[0]
        assert np.array_equal(f[rows], fo)
    else:
        # FP32 decisions: count on the FP32-rounded positions for the sampled rows
        qf = q.astype(np.float32)
        fo = np.array([-(np.sum(qf[r] > qf) - np.sum(qf[r] < qf)) / N for r in rows])
        assert np.array_equal(f[rows], fo)
    s.close()


def test_unsupported_calls_are_rejected():
    """At eps = 0 the sheet force is piecewise constant: no derivatives; no angle,
    so no magnetization."""
    s, _, _ = _sys(100)
    with pytest.raises(MDError):
        s.grad(2)
    with pytest.raises(MDError):
        s.tangent_step(1, np.zeros(100), np.zeros(100))
    with pytest.raises(MDError):
        s.magnetization()

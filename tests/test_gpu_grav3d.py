"""3D self-gravitating model (MD_GRAV3D; not one of the paper's three models)
through the C ABI against the FP64 oracle (needs a GB300).

f_i = -(1/N) sum_j r_ij (|r_ij|^2 + eps)^(-3/2).  Tolerances as for the paper's
models: FP64 |f - f_ora| <= 1e-12 sum_j |f_ij|, FP32 pair arithmetic 2e-5 sum_j |f_ij|;
both the Newton's-third-law (default) and the one-sided kernels.  Sizes span one to
many i-tiles (512 particles) with ragged tails.
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import MDError, System, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-3
SIZES = [1, 2, 3, 33, 511, 512, 513, 1000, 2049, 4097]
KERNEL = {("fp64", 1): 6, ("fp64", 0): 1, ("mixed", 1): 4, ("mixed", 0): 2}


def _sys(N, prec="fp64", symmetric=1, dt=0.01, seed=7):
    s = System(3, N, EPS, dt, seed, precision=prec)
    s.set_tuning("symmetric", symmetric)
    assert s.force_kernel == KERNEL[(prec, symmetric)]
    q, p = inputs.ball_state(N, 1000 + N)
    s.set_state(q, p)
    return s, q, p


def test_device_initial_state_matches_input_generator():
    N = 5000
    with System(3, N, EPS, 0.01, 1234) as s:
        q, p = s.get_state()
    qe, pe = inputs.ball_state(N, 1234)
    np.testing.assert_allclose(q, qe, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(p, pe, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
@pytest.mark.parametrize("N", SIZES)
def test_force_parity(N, prec, tol, symmetric):
    s, q, _ = _sys(N, prec, symmetric)
    f = s.force()
    fo = ora.force(3, q, EPS)
    scale = ora.force_abs(3, q, EPS)
    err = np.abs(f - fo)
    assert np.all(err <= tol * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()
    if N == 1:
        assert np.all(f == 0.0)


@pytest.mark.parametrize("N", [1, 2, 33, 1000, 4097])
def test_fp64_one_step_parity(N):
    dt = 0.01
    s, q0, p0 = _sys(N, dt=dt)
    s.step(1)
    q, p = s.get_state()
    qo, po = ora.step(3, q0, p0, EPS, dt, 1)
    fs = ora.force_abs(3, q0, EPS).max()
    assert np.max(np.abs(q - qo)) <= 1e-12 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-12 * (np.abs(po).max() + dt * fs)


def test_fp64_ten_steps_parity_small():
    dt = 0.01
    s, q0, p0 = _sys(33, dt=dt)
    s.step(4)
    s.step(6)  # two calls: the first-same-as-last force cache
    q, p = s.get_state()
    qo, po = ora.step(3, q0, p0, EPS, dt, 10)
    assert np.max(np.abs(q - qo)) <= 1e-11 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-11 * max(1.0, np.abs(po).max())


@pytest.mark.parametrize("N", [1, 2, 33, 1000, 4097])
def test_energy_parity(N):
    s, q, p = _sys(N)
    K, V = s.energy()
    assert abs(K - ora.kinetic(p)) <= 1e-12 * max(abs(K), 1e-300)
    Vo = ora.potential(3, q, EPS)
    assert abs(V - Vo) <= 1e-12 * max(abs(Vo), 1.0), (V, Vo)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_momentum_and_angular_momentum_conserved(prec):
    N = 4097
    s, q0, p0 = _sys(N, prec)
    s.step(20)
    q, p = s.get_state()
    for c in range(3):
        drift = abs(p[c * N:(c + 1) * N].sum() - p0[c * N:(c + 1) * N].sum())
        assert drift < (1e-12 if prec == "fp64" else 1e-6) * np.abs(p0).sum(), drift

    def L(q, p):
        return np.cross(q.reshape(3, N).T, p.reshape(3, N).T).sum(axis=0)

    scale = np.sum(np.abs(q0)) * np.abs(p0).max()
    assert np.max(np.abs(L(q, p) - L(q0, p0))) < (1e-12 if prec == "fp64" else 1e-6) * scale


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_runs_are_bitwise_deterministic(prec):
    out = []
    for _ in range(2):
        s, _, _ = _sys(3000, prec)
        s.step(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_mixed_energy_error_within_twice_fp64():
    res = {}
    for prec in ("fp64", "mixed"):
        s, _, _ = _sys(2048, prec, dt=0.005)
        e0 = sum(s.energy())
        worst = 0.0
        for _ in range(10):
            s.step(10)
            worst = max(worst, abs((sum(s.energy()) - e0) / e0))
        res[prec] = worst
    assert res["mixed"] <= 2 * res["fp64"] + 1e-9, res


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_sampled_force_parity(prec):
    N = 131072
    s = System(3, N, EPS, 0.01, 45, precision=prec)
    q, _ = s.get_state()
    f = s.force().reshape(3, N)
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(9, np.arange(62)) % np.uint64(N)]).astype(np.int64))
    fo, scale = ora.force_rows(3, q, rows, EPS, with_abs=True)
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.all(np.abs(f[:, rows] - fo) <= tol * scale), (np.abs(f[:, rows] - fo) / scale).max()
    s.close()


def test_unsupported_calls_are_rejected():
    """The magnetization (and its gradient) needs an angle; the disk recipe is the
    2D model's.  Gradients of the kinetic energy are supported."""
    s, q, p = _sys(100)
    with pytest.raises(MDError):
        s.grad(2, 1)
    with pytest.raises(MDError):
        s.magnetization()
    with pytest.raises(MDError):
        s.set_ic(2)  # the disk recipe is for the 2D model
    s.set_ic(5, [0.1], seed=3)  # the ball recipe
    q2, p2 = s.get_state()
    qe, pe = inputs.ball_state(100, 3, sigma=0.1)
    np.testing.assert_allclose(q2, qe, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(p2, pe, rtol=1e-14, atol=1e-15)

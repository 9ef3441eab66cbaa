"""md_grad (discrete adjoint through the C ABI) against the oracle's discrete
adjoint and against central finite differences of the GPU forward map.

Tolerances: FP64 gradient vs the oracle's gradient 1e-10 relative (max over
components, relative to the largest component); directional central
differences at N = 1,024 (2D, the config's size) 1e-6 relative.
"""
import numpy as np
import pytest
import torch

import oracle as ora
from paper_1212_0262_gb300 import System, inputs
from paper_1212_0262_gb300.autograd import rollout

pytestmark = pytest.mark.gpu

EPS = {0: 0.0, 1: 0.01, 2: 1e-3, 3: 1e-2, 4: 0.05}
DT = {0: 0.1, 1: 0.05, 2: 0.01, 3: 0.01, 4: 0.01}


def _sys(model, N, prec="fp64", seed=3):
    s = System(model, N, EPS[model], DT[model], 1, precision=prec)
    q, p = inputs.default_state(model, N, seed)
    s.set_state(q, p)
    return s, q, p


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("model,obs", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (3, 0), (4, 0)])
@pytest.mark.parametrize("N,nsteps,K", [(64, 20, 7), (257, 9, 3)])
def test_fp64_gradient_matches_oracle_adjoint(model, obs, N, nsteps, K):
    s, q, p = _sys(model, N)
    val, gq, gp, ge = s.grad(nsteps, obs, K)
    ov, oq, op, oe = ora.grad(model, q, p, EPS[model], DT[model], nsteps, obs)
    assert abs(val - ov) <= 1e-12 * abs(ov)
    assert _rel(gq, oq) <= 1e-10, _rel(gq, oq)
    assert _rel(gp, op) <= 1e-10, _rel(gp, op)
    if model != 0:
        assert abs(ge - oe) <= 1e-10 * max(abs(oe), 1e-300)


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_state_is_unchanged_and_checkpoint_interval_does_not_matter(model):
    s, q, p = _sys(model, 300)
    g1 = s.grad(12, 0, 1)
    q1, p1 = s.get_state()
    assert np.array_equal(q1, q) and np.array_equal(p1, p)
    g2 = s.grad(12, 0, 100)
    for a, b in zip(g1[1:3], g2[1:3]):
        assert _rel(a, b) <= 1e-11
    # and a plain forward from the same state still matches md_step
    s.step(12)
    assert abs(s.energy()[0] - g1[0]) <= 1e-13 * abs(g1[0])


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_zero_steps_gives_the_terminal_adjoint(model):
    s, q, p = _sys(model, 100)
    val, gq, gp, ge = s.grad(0, 0, 5)
    assert np.array_equal(gp, p) and not gq.any() and ge == 0.0


def _fd_observable(s, q, p, eps, nsteps, obs):
    s.set_state(q, p)
    if eps is not None:
        s._chk(__import__("paper_1212_0262_gb300").binding.load().md_set_eps(s._h, eps))
    s.step(nsteps)
    if obs == 0:
        return s.energy()[0]
    mx, my = s.magnetization()
    return float(np.hypot(mx, my))


@pytest.mark.parametrize("model,N,nsteps,obs", [(2, 1024, 100, 0), (1, 1024, 40, 0), (1, 512, 40, 1),
                                                (0, 4096, 40, 1), (3, 1024, 60, 0), (4, 1024, 60, 0)])
def test_gradient_matches_central_differences(model, N, nsteps, obs):
    """Directional derivatives along seeded random directions, and d/d eps."""
    s, q, p = _sys(model, N, seed=11)
    val, gq, gp, ge = s.grad(nsteps, obs, 20)
    h = 1e-6
    for k in range(3):
        dq = inputs.uniform(100 + k, 0, q.size) - 0.5
        dp = inputs.uniform(200 + k, 0, p.size) - 0.5
        up = _fd_observable(s, q + h * dq, p + h * dp, None, nsteps, obs)
        dn = _fd_observable(s, q - h * dq, p - h * dp, None, nsteps, obs)
        fd = (up - dn) / (2 * h)
        ad = float(np.dot(gq, dq) + np.dot(gp, dp))
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), abs(fd)), (k, fd, ad)
    if model != 0:
        e = EPS[model]
        he = 1e-6 * e
        up = _fd_observable(s, q, p, e + he, nsteps, obs)
        dn = _fd_observable(s, q, p, e - he, nsteps, obs)
        fde = (up - dn) / (2 * he)
        assert abs(fde - ge) <= 1e-6 * max(abs(ge), abs(fde)), (fde, ge)


@pytest.mark.parametrize("model", [1, 2, 3, 4])
def test_mixed_gradient_close_to_fp64(model):
    s, q, p = _sys(model, 2048)
    ref = s.grad(20, 0, 5)
    m, _, _ = _sys(model, 2048, "mixed")
    mix = m.grad(20, 0, 5)
    assert _rel(mix[1], ref[1]) < 1e-3 and _rel(mix[2], ref[2]) < 1e-3
    assert abs(mix[3] - ref[3]) < 1e-3 * abs(ref[3])


def test_autograd_function_backward():
    s, q, p = _sys(2, 256)
    q0 = torch.tensor(q, requires_grad=True)
    p0 = torch.tensor(p, requires_grad=True)
    eps = torch.tensor(EPS[2], dtype=torch.float64, requires_grad=True)
    out = rollout(q0, p0, eps, s, 10, 0, 4)
    (3.0 * out).backward()
    val, gq, gp, ge = s.grad(10, 0, 4)
    assert abs(out.item() - val) <= 1e-14 * abs(val)
    np.testing.assert_allclose(q0.grad.numpy(), 3.0 * gq, rtol=0, atol=0)
    np.testing.assert_allclose(p0.grad.numpy(), 3.0 * gp, rtol=0, atol=0)
    assert eps.grad.item() == 3.0 * ge


@pytest.mark.parametrize("N", [1, 3, 1000, 1025, 2049])
@pytest.mark.parametrize("model", [3, 4])
def test_fp64_gradient_ragged_sizes(model, N):
    """The 3D and sheet reverse-stage kernels across one to several i-tiles with
    ragged tails (padding records far away, lambda_p = 0)."""
    s, q, p = _sys(model, N, seed=5)
    val, gq, gp, ge = s.grad(5, 0, 2)
    ov, oq, op, oe = ora.grad(model, q, p, EPS[model], DT[model], 5, 0)
    assert _rel(gq, oq) <= 1e-10 and _rel(gp, op) <= 1e-10
    assert abs(ge - oe) <= 1e-10 * max(abs(oe), 1e-300) + 1e-300


def test_reverse_stages_refuse_what_has_no_derivative():
    """Sheets at eps = 0 (a piecewise-constant force) and the magnetization of the
    models without an angle: MD_EINVAL with a message, the context still usable."""
    s = System(4, 100, 0.0, 0.01, 1)
    with pytest.raises(RuntimeError, match="eps > 0"):
        s.grad(3, 0, 2)
    with pytest.raises(RuntimeError, match="eps > 0"):
        s.tangent_step(1, np.zeros(100), np.zeros(100))
    s.step(1)
    for model in (2, 3, 4):
        t, _, _ = _sys(model, 64)
        with pytest.raises(RuntimeError, match="HMF and Ring"):
            t.grad(3, 1, 2)


@pytest.mark.parametrize("model", [1, 2, 3])
def test_rollout_by_model_matches_md_grad(model):
    """rollout_model(q0, p0, eps, model, nsteps, dt): the context is made for the call;
    value and gradients equal md_grad on the same state."""
    from paper_1212_0262_gb300.autograd import rollout_model

    N = 300
    s, q, p = _sys(model, N)
    val, gq, gp, ge = s.grad(8, 0, 3)
    q0 = torch.tensor(q, requires_grad=True)
    p0 = torch.tensor(p, requires_grad=True)
    eps = torch.tensor(EPS[model], dtype=torch.float64, requires_grad=True)
    out = rollout_model(q0, p0, eps, model, 8, DT[model], 0, checkpoint_every=3)
    out.backward()
    assert out.item() == val
    assert np.array_equal(q0.grad.numpy(), gq) and np.array_equal(p0.grad.numpy(), gp)
    assert eps.grad.item() == ge


def _duality(s, nsteps, K, seed):
    """<grad K(T), v> and <p(T), dp(T)>, dp carried from v by md_tangent_step, with the
    scale sum |terms| of the larger side (the state is advanced to T)."""
    q, _ = s.get_state()
    n = q.size
    _, gq, gp, _ = s.grad(nsteps, 0, K)
    vq = inputs.uniform(seed, 0, n) - 0.5
    vp = inputs.uniform(seed + 1, 0, n) - 0.5
    _, dp = s.tangent_step(nsteps, vq, vp)
    _, pT = s.get_state()
    lhs, rhs = gq @ vq + gp @ vp, pT @ dp
    scale = max(np.abs(gq * vq).sum() + np.abs(gp * vp).sum(), np.abs(pT * dp).sum())
    return lhs, rhs, scale


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_fp64_adjoint_is_the_transpose_of_the_tangent(model):
    """The reverse sweep is the transpose of the forward derivative of the same step
    map: <grad_x0 K(T), v> = <dK/dx(T), dx(T)> = <p(T), dp(T)> for K = sum p^2 / 2,
    with the gradient rebuilt from checkpoints and the tangent carried forward (several
    tiles with a ragged tail)."""
    s, _, _ = _sys(model, 5000)
    lhs, rhs, scale = _duality(s, 12, 5, 31)
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)
    s.close()


def test_full_size_mixed_adjoint_is_the_transpose_of_the_tangent():
    """The benchmark's gradient (2D, N = 262,144, eps = 1e-4, dt = 0.01, 100 steps,
    checkpoints every 20 steps, mixed precision) and a tangent run along a seeded
    direction agree as the transpose of each other, within the mixed path's rounding."""
    with System(2, 262_144, 1e-4, 0.01, 4, precision="mixed") as s:
        lhs, rhs, scale = _duality(s, 100, 20, 41)
    assert abs(lhs - rhs) <= 1e-4 * scale, (lhs, rhs, scale, abs(lhs - rhs) / scale)

"""md_tangent_step (forward-mode derivative of md_step's map) against central
differences of the oracle's step, and the Lyapunov estimate built on it."""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs

pytestmark = pytest.mark.gpu

EPS = {0: 0.0, 1: 0.01, 2: 1e-3, 3: 1e-2, 4: 0.05}
DT = {0: 0.1, 1: 0.05, 2: 0.01, 3: 0.01, 4: 0.01}


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_tangent_matches_oracle_central_differences(model):
    N, nsteps = 200, 12
    q0, p0 = inputs.default_state(model, N, 13)
    n = q0.size
    dq0 = inputs.uniform(21, 0, n) - 0.5
    dp0 = inputs.uniform(22, 0, n) - 0.5
    with System(model, N, EPS[model], DT[model], 1, precision="fp64") as s:
        s.set_state(q0, p0)
        dq, dp = s.tangent_step(nsteps, dq0, dp0)
        q, p = s.get_state()
    qo, po = ora.step(model, q0, p0, EPS[model], DT[model], nsteps)
    assert np.max(np.abs(q - qo)) <= 1e-12 * max(1.0, np.abs(qo).max())
    h = 1e-6
    qa, pa = ora.step(model, q0 + h * dq0, p0 + h * dp0, EPS[model], DT[model], nsteps)
    qb, pb = ora.step(model, q0 - h * dq0, p0 - h * dp0, EPS[model], DT[model], nsteps)
    fq, fp = (qa - qb) / (2 * h), (pa - pb) / (2 * h)
    scale = max(np.abs(fq).max(), np.abs(fp).max())
    assert np.max(np.abs(dq - fq)) <= 1e-6 * scale and np.max(np.abs(dp - fp)) <= 1e-6 * scale


@pytest.mark.parametrize("model", [1, 2, 3, 4])
def test_mixed_tangent_close_to_fp64(model):
    N = 1024
    q0, p0 = inputs.default_state(model, N, 5)
    d = inputs.uniform(6, 0, 2 * q0.size) - 0.5
    out = {}
    for prec in ("fp64", "mixed"):
        with System(model, N, EPS[model], DT[model], 1, precision=prec) as s:
            s.set_state(q0, p0)
            out[prec] = s.tangent_step(10, d[:q0.size], d[q0.size:])
    for a, b in zip(out["mixed"], out["fp64"]):
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b))


def test_lyapunov_estimate_is_positive_and_stable_hmf():
    """HMF water-bag (chaotic): the estimate is positive and barely depends on
    how often the tangent is renormalised."""
    vals = []
    for every in (5, 20):
        with System(0, 5000, 0.0, 0.1, 3) as s:
            vals.append(s.lyapunov(400, every, seed=1))
    assert vals[0] > 0.0 and abs(vals[0] - vals[1]) <= 1e-6 * abs(vals[0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_device_lyapunov_equals_the_host_renormalisation_loop(model, prec):
    """md_lyapunov (tangent kept on the device, renormalised there) against the same
    estimate made on the host around md_tangent_step (pinned above to central
    differences of the oracle): the same state afterwards, bit for bit, and the same
    sum of log norms to rounding; 37 steps in blocks of 10 (a shorter last block)."""
    N, nsteps, every = 500, 37, 10
    q0, p0 = inputs.default_state(model, N, 4)
    n = q0.size
    d = inputs.uniform(3, 0, 2 * n) - 0.5
    with System(model, N, EPS[model], DT[model], 1, precision=prec) as a:
        a.set_state(q0, p0)
        lam = a.lyapunov(nsteps, every, seed=3)
        qa, pa = a.get_state()
    with System(model, N, EPS[model], DT[model], 1, precision=prec) as b:
        b.set_state(q0, p0)
        v = d / np.linalg.norm(d)
        dq, dp = v[:n], v[n:]
        total, done = 0.0, 0
        while done < nsteps:
            k = min(every, nsteps - done)
            dq, dp = b.tangent_step(k, dq, dp)
            norm = float(np.sqrt(np.dot(dq, dq) + np.dot(dp, dp)))
            total += np.log(norm)
            dq, dp = dq / norm, dp / norm
            done += k
        qb, pb = b.get_state()
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    ref = total / (nsteps * DT[model])
    assert abs(lam - ref) <= 1e-9 * abs(ref), (lam, ref)

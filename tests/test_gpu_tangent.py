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

"""One fused integrator stage at the benchmark sizes (kick with the force at the
current positions, then drift; Sec. 3 step list with the Eq. 4 coefficients),
through md_stage, checked on sampled particles against the oracle's direct force
sums.  The stage kernels are the ones md_step replays from its CUDA graphs
(test_step_graphs_match_stage_by_stage shows the two bitwise equal), so this
covers the fused epilogue of every model at the size the benchmark times.

Tolerances: p1 = p0 + b dt f(q0) within |b dt| * (1e-12 FP64, 2e-5 mixed) *
sum_j |f_ij| plus 4 ulp of the operands; q1 = q0 + d dt p1 within 4 ulp (the
drift is a single FP64 multiply-add on the GPU's own p1).  The 1D-sheet force at
eps = 0 is a count of signs and is exact: FP64 signs on the FP64 positions, FP32
signs on the FP32-rounded positions for the mixed path.
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs
from paper_1212_0262_gb300.system import yoshida

pytestmark = pytest.mark.gpu

U = np.finfo(np.float64).eps

# model, N, eps, dt, seed: the benchmark's single-system workloads
WORKLOADS = [(0, 50_000_000, 0.0, 0.1, 2), (1, 131_072, 0.01, 0.05, 3), (2, 262_144, 1e-4, 0.01, 4),
             (3, 131_072, 1e-3, 0.01, 5), (4, 262_144, 0.0, 0.01, 6)]


def _rows(N):
    return np.unique(np.concatenate([[0, 1, N - 1], inputs.splitmix64(21, np.arange(61)) % np.uint64(N)]).astype(np.int64))


def _sheet_counts(q, rows, mixed):
    x = q.astype(np.float32) if mixed else q
    N = q.size
    return np.array([-(np.sum(x[r] > x) - np.sum(x[r] < x)) / N for r in rows])[None, :]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("model,N,eps,dt,seed", WORKLOADS)
def test_full_size_stage_sampled(model, N, eps, dt, seed, prec):
    B0, B1, D0, D1 = yoshida()
    # (B1, D1): D1 = w0 < 0, so the drift runs backwards and its sign is checked too
    b, d = B1, D1
    with System(model, N, eps, dt, seed, precision=prec) as s:
        q0, p0 = s.get_state()
        s.stage(b, d)
        q1, p1 = s.get_state()
    dim = q0.size // N
    rows = _rows(N)
    if model == 4:
        f = _sheet_counts(q0, rows, prec == "mixed")
        scale = np.zeros_like(f)
    else:
        f, scale = ora.force_rows(model, q0, rows, eps, with_abs=True)
    tol = 1e-12 if prec == "fp64" else 2e-5
    for c in range(dim):
        idx = c * N + rows
        kick = b * dt * f[c]
        p_exp = p0[idx] + kick
        bound_p = abs(b * dt) * tol * scale[c] + 4 * U * (np.abs(p0[idx]) + np.abs(kick))
        err_p = np.abs(p1[idx] - p_exp)
        assert np.all(err_p <= bound_p), (c, (err_p / np.maximum(bound_p, 1e-300)).max())
        drift = d * dt * p1[idx]
        q_exp = q0[idx] + drift
        err_q = np.abs(q1[idx] - q_exp)
        assert np.all(err_q <= 4 * U * (np.abs(q0[idx]) + np.abs(drift))), (c, err_q.max())
    # particles not sampled moved too (the whole state went through the stage)
    assert not np.array_equal(p1, p0) and not np.array_equal(q1, q0)

"""Largest sizes: HMF with particle indices past the 32-bit range, and the pair
models at the paper's largest N = 10^6 (Sec. 4; ragged: N = 10^6 + 3) in their
default kernels.

HMF at N = 2^31 + 1001 holds 34 GB of state (plus as much again for the device
copies the test makes).  Its input theta_i = alpha i has the closed-form
magnetization (Eq. 7) M = e^{i alpha (N-1)/2} sin(alpha N / 2) / (N sin(alpha / 2)),
so the check needs no O(N) host pass: md_magnetization against the closed form,
then one kick-drift stage from p = 0 on sampled particles (indices 2^31 - 1, 2^31,
2^31 + 1 and N - 1 among them) against p1 = b dt (cos th My - sin th Mx) (Eq. 6),
the closed form and the force's sign convention being pinned to the oracle in
test_oracle.py (test_hmf_closed_form_magnetization_of_an_arithmetic_progression).
"""
import numpy as np
import pytest
import torch

import oracle as ora
from paper_1212_0262_gb300 import System, inputs
from paper_1212_0262_gb300.system import yoshida

pytestmark = pytest.mark.gpu

U = np.finfo(np.float64).eps


def _closed_form_m(alpha, N):
    amp = np.sin(alpha * N / 2.0) / (N * np.sin(alpha / 2.0))
    return np.cos(alpha * (N - 1) / 2.0) * amp, np.sin(alpha * (N - 1) / 2.0) * amp


def _hmf_force(th, mx, my):
    return np.cos(th) * my - np.sin(th) * mx


@pytest.mark.parametrize("prec,tol_m,tol_f", [("fp64", 1e-12, 1e-12), ("mixed", 1e-12, 2e-6)])
def test_hmf_beyond_32_bit_particle_indices(prec, tol_m, tol_f):
    N = 2**31 + 1001
    alpha = 2.5e-9  # theta spans [0, 5.37): the sums do not cancel
    B0, B1, D0, D1 = yoshida()
    dt = 0.1
    with System(0, N, 0.0, dt, 1, precision=prec) as s:
        th = torch.arange(N, dtype=torch.float64, device="cuda").mul_(alpha)
        p = torch.zeros(N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # the copies below run on the context's own stream
        s.set_state_device(th.data_ptr(), p.data_ptr())
        mx, my = s.magnetization()
        ex, ey = _closed_form_m(alpha, N)
        assert abs(mx - ex) <= tol_m and abs(my - ey) <= tol_m, (mx - ex, my - ey)
        s.stage(B0, D0)
        s.get_state_device(th.data_ptr(), p.data_ptr())
        torch.cuda.synchronize()
        rows = np.unique(np.concatenate([[0, 1, 2**31 - 1, 2**31, 2**31 + 1, N - 2, N - 1],
                                         inputs.splitmix64(77, np.arange(57)) % np.uint64(N)]).astype(np.int64))
        idx = torch.from_numpy(rows).cuda()
        th1, p1 = th[idx].cpu().numpy(), p[idx].cpu().numpy()
    th0 = alpha * rows.astype(np.float64)
    kick = B0 * dt * _hmf_force(th0, ex, ey)
    # kick: the force's error (M and the per-particle sine/cosine) times |b dt|
    assert np.all(np.abs(p1 - kick) <= abs(B0 * dt) * tol_f + 4 * U * np.abs(kick)), np.abs(p1 - kick).max()
    # drift from the GPU's own p1, on top of the FP64 rounding of theta_i = alpha i
    drift = D0 * dt * p1
    assert np.all(np.abs(th1 - (th0 + drift)) <= 8 * U * (np.abs(th0) + np.abs(drift)))
    del th, p
    torch.cuda.empty_cache()


@pytest.mark.parametrize("model,eps", [(1, 0.01), (2, 1e-4)])
def test_pairs_at_the_papers_largest_n(model, eps):
    """N = 10^6 + 3 (ragged against every tile size) in the default mixed kernel,
    which is the Newton's-third-law form at this size: forces on sampled particles
    against the oracle's direct sums."""
    N = 1_000_003
    with System(model, N, eps, 0.01, 8, precision="mixed") as s:
        assert s.force_kernel in (4, 5), s.force_kernel  # MD_KERNEL_PAIRS_SYM, MD_KERNEL_PAIRS_TC_SYM
        q, _ = s.get_state()
        f = s.force().reshape(2 if model == 2 else 1, N)
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(19, np.arange(30)) % np.uint64(N)]).astype(np.int64))
    fo, scale = ora.force_rows(model, q, rows, eps, with_abs=True)
    assert np.all(np.abs(f[:, rows] - fo) <= 2e-5 * scale), (np.abs(f[:, rows] - fo) / scale).max()

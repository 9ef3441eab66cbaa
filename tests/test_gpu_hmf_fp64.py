"""The FP64 HMF stages take the cosine and sine of every new angle from a
table-driven reduction (theta = k pi/2048 + r, a 4096-entry table of (sin, cos)(k pi/2048),
Taylor terms in r, the index k and the terms below 2^-33 in FP32; from |theta| = 2^20 on
the CUDA sincos).  Their accuracy is pinned here against the oracle's libm sin and cos
through the HMF force of Eq. 6: within 2e-15 of sum_j |f_ij| (a few units in the last
place of every cosine and sine, far inside the 1e-12 parity bound), for angles spread
over up to +-2e9, on both sides of 2^20."""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs

pytestmark = pytest.mark.gpu

TOL = 2e-15


@pytest.mark.parametrize("span", [1.0, 3.2, 1e3, 1e6, 1.0485e6, 1.2e6, 2e9])
def test_fp64_hmf_force_from_table_sine_cosine(span):
    N = 4099
    q = (inputs.uniform(31, 0, N) * 2.0 - 1.0) * span
    p = inputs.uniform(32, 0, N) * 2.4 - 1.2
    with System(0, N, 0.0, 0.1, 1) as s:
        s.set_state(q, p)
        f = s.force()  # (cos, sin) of the current angles from the priming pass
        fo = ora.force(0, q)
        scale = ora.force_abs(0, q)
        assert np.all(np.abs(f - fo) <= TOL * scale), (np.abs(f - fo) / scale).max()
        s.stage(0.6756, 1.3512)  # one fused stage: the new angles' (cos, sin) from the stage kernel
        q1, p1 = s.get_state()
        f1 = s.force()
        fo1 = ora.force(0, q1)
        scale1 = ora.force_abs(0, q1)
        assert np.all(np.abs(f1 - fo1) <= TOL * scale1), (np.abs(f1 - fo1) / scale1).max()


def test_fp64_hmf_table_at_the_table_points():
    """Angles on the table grid k pi/2048 (r = 0 up to the reduction's rounding) and
    half way between (|r| = pi/4096, the largest; the index k of either neighbour), over
    more than one turn both ways, and the same near the end of the table range (2^20)."""
    k = np.arange(-5200, 5200, dtype=np.float64)
    kb = np.floor(2.0**20 / (np.pi / 2048)) - np.arange(0, 3000, dtype=np.float64)
    k = np.concatenate([k, kb, -kb])
    q = np.concatenate([k * (np.pi / 2048), (k + 0.5) * (np.pi / 2048)])
    N = q.size
    with System(0, N, 0.0, 0.1, 1) as s:
        s.set_state(q, np.zeros(N))
        f = s.force()
    fo = ora.force(0, q)
    scale = ora.force_abs(0, q)
    assert np.all(np.abs(f - fo) <= TOL * scale), (np.abs(f - fo) / scale).max()

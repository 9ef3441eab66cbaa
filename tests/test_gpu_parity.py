"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300).

Tolerances:
  FP64 forces   |f_gpu - f_ora| <= 1e-12 * sum_j |f_ij|   (per particle and
                component; the summation-order bound, since plain relative error is
                ill-conditioned where the pair forces cancel)
  FP64 one step |dq| <= 1e-12 max(1, |q|_inf), |dp| <= 1e-12 (|p|_inf + dt |sum_j |f_ij||_inf)
  mixed forces  |f_mix - f_ora| <= 2e-5 * sum_j |f_ij|  (FP32 pair arithmetic and
                FP32 positions; the FP64 state is exact)
  energies      1e-12 relative (FP64 reductions)
"""
import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import System, inputs

pytestmark = pytest.mark.gpu

EPS = {0: 0.0, 1: 0.01, 2: 1e-3}
SIZES = [1, 2, 3, 31, 32, 33, 1000, 1024, 4097]


def _sys(model, N, prec="fp64", dt=0.05, seed=7):
    s = System(model, N, EPS[model], dt, seed, precision=prec)
    q, p = inputs.default_state(model, N, 1000 + N)
    s.set_state(q, p)
    return s, q, p


def _force_err(model, q, f_gpu):
    f_ora = ora.force(model, q, EPS[model])
    scale = ora.force_abs(model, q, EPS[model])
    err = np.abs(f_gpu - f_ora)
    return err, scale, f_ora


# ------------------------------------------------------------------ IC ----

@pytest.mark.parametrize("model", [0, 1, 2])
def test_device_initial_state_matches_input_generator(model):
    N = 5000
    with System(model, N, EPS[model] or 0.0, 0.1, 1234) as s:
        q, p = s.get_state()
    qe, pe = inputs.default_state(model, N, 1234)
    if model == 0:
        assert np.array_equal(q, qe) and np.array_equal(p, pe)
    elif model == 1:
        assert np.array_equal(q, qe)
        np.testing.assert_allclose(p, pe, rtol=1e-14, atol=1e-15)
    else:
        np.testing.assert_allclose(q, qe, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(p, pe, rtol=1e-14, atol=1e-15)


# --------------------------------------------------------------- forces ---

@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_force_parity(model, N, symmetric):
    """FP64 forces; Ring and 2D both with every unordered pair once (default) and
    with every ordered pair (the one-sided kernel)."""
    if model == 0 and symmetric == 0:
        pytest.skip("HMF has no pair kernel")
    s, q, p = _sys(model, N)
    s.set_tuning("symmetric", symmetric)
    if model:
        assert s.force_kernel == (6 if symmetric else 1)
    f = s.force()
    err, scale, f_ora = _force_err(model, q, f)
    assert np.all(err <= 1e-12 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()
    if N == 1:
        assert np.all(f == 0.0)


# FP32 pair-kernel variants: (ring_tc, symmetric); the default is (1, 1)
VARIANTS = {"default": None, "one_sided_cuda_cores": (0, 0), "one_sided_tensor_cores": (1, 0)}


def _variant(s, name):
    if VARIANTS[name] is not None:
        s.set_tuning("ring_tc", VARIANTS[name][0])
        s.set_tuning("symmetric", VARIANTS[name][1])
    return s


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("model", [0, 1, 2])
def test_mixed_force_error_bound(model, N, variant):
    if model == 0 and variant != "default":
        pytest.skip("HMF has no pair kernel")
    s, q, p = _sys(model, N, "mixed")
    f = _variant(s, variant).force()
    err, scale, _ = _force_err(model, q, f)
    assert np.all(err <= 2e-5 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()


# ---------------------------------------------------------- integration ---

@pytest.mark.parametrize("N", [1, 2, 33, 1000, 4097])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_one_step_parity(model, N):
    dt = 0.05
    s, q0, p0 = _sys(model, N, dt=dt)
    s.step(1)
    q, p = s.get_state()
    qo, po = ora.step(model, q0, p0, EPS[model], dt, 1)
    fs = ora.force_abs(model, q0, EPS[model]).max()
    assert np.max(np.abs(q - qo)) <= 1e-12 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-12 * (np.abs(po).max() + dt * fs)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_ten_steps_parity_small(model):
    dt = 0.02
    s, q0, p0 = _sys(model, 33, dt=dt)
    s.step(4)
    s.step(6)  # two calls: exercises the first-same-as-last force cache
    q, p = s.get_state()
    qo, po = ora.step(model, q0, p0, EPS[model], dt, 10)
    assert np.max(np.abs(q - qo)) <= 1e-11 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-11 * max(1.0, np.abs(po).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_runs_are_bitwise_deterministic(model, prec):
    out = []
    for _ in range(2):
        s, _, _ = _sys(model, 3000, prec)
        s.step(3)
        out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_total_momentum_conserved(model, prec):
    N = 4097
    s, q0, p0 = _sys(model, N, prec)
    s.step(20)
    q, p = s.get_state()
    d = 2 if model == 2 else 1
    for c in range(d):
        drift = abs(p[c * N:(c + 1) * N].sum() - p0[c * N:(c + 1) * N].sum())
        assert drift < (1e-12 if prec == "fp64" else 1e-6) * np.abs(p0).sum(), drift


# ---------------------------------------------------------- observables ---

@pytest.mark.parametrize("N", [1, 2, 33, 1000, 4097])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_energy_parity(model, N):
    s, q, p = _sys(model, N)
    K, V = s.energy()
    assert abs(K - ora.kinetic(p)) <= 1e-12 * max(abs(K), 1e-300)
    Vo = ora.potential(model, q, EPS[model])
    assert abs(V - Vo) <= 1e-12 * max(abs(Vo), 1.0), (V, Vo)


@pytest.mark.parametrize("eps", [1e-3, 1e-14])
def test_2d_potential_over_a_wide_range_of_separations(eps):
    """The 2D potential takes each thread row's logarithms as the logarithm of a
    renormalised product.  Radii log-uniform in [1e-7, 1e5] (factors s = r^2 + eps
    over 24 decades, products far outside the double range) keep the bound, taken
    against sum_{i<j} |log s_ij| / N since the logarithms have both signs."""
    N = 3000
    u = inputs.uniform(51, 0, 2 * N)
    rad = 10.0 ** (-7.0 + 12.0 * u[:N])
    ang = 2.0 * np.pi * u[N:]
    q = np.concatenate([rad * np.cos(ang), rad * np.sin(ang)])
    with System(2, N, eps, 0.01, 1, precision="fp64") as s:
        s.set_state(q, np.zeros_like(q))
        _, V = s.energy()
    Vo = ora.potential(2, q, eps)
    x, y = q[:N], q[N:]
    scale = sum(np.abs(np.log((x[i] - x[i + 1:]) ** 2 + (y[i] - y[i + 1:]) ** 2 + eps)).sum() for i in range(N)) / N
    assert abs(V - Vo) <= 1e-12 * scale, (V, Vo, scale)


@pytest.mark.parametrize("model", [0, 1])
def test_magnetization_parity(model):
    s, q, p = _sys(model, 10001)
    mx, my = s.magnetization()
    ox, oy = ora.magnetization(q)
    assert abs(mx - ox) < 1e-13 and abs(my - oy) < 1e-13


def test_mixed_energy_error_within_twice_fp64():
    """Long run judged by the relative energy error (Sec. 4): the mixed path's
    stays within twice the FP64 path's (plus a floor at FP64 resolution)."""
    res = {}
    for model, N, dt, nst in ((1, 2048, 0.05, 100), (2, 2048, 0.01, 100), (0, 100000, 0.1, 100)):
        for prec in ("fp64", "mixed"):
            s, q, p = _sys(model, N, prec, dt=dt)
            e0 = sum(s.energy())
            worst = 0.0
            for _ in range(10):
                s.step(nst // 10)
                worst = max(worst, abs((sum(s.energy()) - e0) / e0))
            res[(model, prec)] = worst
        assert res[(model, "mixed")] <= 2 * res[(model, "fp64")] + 1e-12, res


# ------------------------------------------------ full-size sampled checks --

@pytest.mark.parametrize("prec", ["mixed", "fp64", "mixed_one_sided", "fp64_one_sided"])
@pytest.mark.parametrize("model,N,eps", [(0, 50_000_000, 0.0), (1, 131072, 0.01), (2, 262144, 1e-4)])
def test_full_size_sampled_force_parity(model, N, eps, prec):
    """Bench-size systems in the bench's launch configuration: forces on 64
    sampled particles against the oracle's direct sums."""
    if model == 0 and prec.endswith("one_sided"):
        pytest.skip("HMF has no pair kernel")
    s = System(model, N, eps, 0.05, 42 + model, precision=prec.split("_")[0])
    if prec.endswith("one_sided"):
        _variant(s, "one_sided_cuda_cores")
    q, _ = s.get_state()
    f = s.force().reshape(2 if model == 2 else 1, N)
    rows = np.unique(np.concatenate([[0, N - 1], inputs.splitmix64(9, np.arange(62)) % np.uint64(N)]).astype(np.int64))
    fo, scale = ora.force_rows(model, q, rows, eps, with_abs=True)
    tol = 1e-12 if prec.startswith("fp64") else 2e-5
    assert np.all(np.abs(f[:, rows] - fo) <= tol * scale), (np.abs(f[:, rows] - fo) / scale).max()
    s.close()


@pytest.mark.parametrize("tc", [1, 2])
@pytest.mark.parametrize("N", [1, 2, 33, 1000, 4097])
def test_ring_tensor_core_force_error_bound(N, tc):
    """Ring FP32 path with sin(d) and sin(d/2) from split-TF32 tensor-core MMAs."""
    s, q, p = _sys(1, N, "mixed")
    s.set_tuning("ring_tc", tc)
    s.set_tuning("symmetric", 0)
    f = s.force()
    err, scale, _ = _force_err(1, q, f)
    assert np.all(err <= 2e-5 * scale + 1e-300), (err / np.maximum(scale, 1e-300)).max()
    if N == 1:
        assert f[0] == 0.0


@pytest.mark.parametrize("tc", [1, 2])
def test_ring_tensor_core_steps_match_fp32_kernel(tc):
    """Ten steps with the tensor-core kernel stay as close to FP64 as the FP32
    kernel, and the energy error keeps the mixed-vs-FP64 bound."""
    N, dt = 3000, 0.05
    ref, q0, p0 = _sys(1, N, "fp64", dt=dt)
    tcs, _, _ = _sys(1, N, "mixed", dt=dt)
    tcs.set_tuning("ring_tc", tc)
    tcs.set_tuning("symmetric", 0)
    e0 = sum(ref.energy())
    ref.step(10)
    tcs.step(10)
    (qr, pr), (qt, pt_) = ref.get_state(), tcs.get_state()
    assert np.max(np.abs(qt - qr)) < 1e-5 and np.max(np.abs(pt_ - pr)) < 1e-5
    d_ref = abs(sum(ref.energy()) - e0) / abs(e0)
    d_tc = abs(sum(tcs.energy()) - e0) / abs(e0)
    assert d_tc <= 2 * d_ref + 1e-9, (d_tc, d_ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_step_graphs_match_stage_by_stage(model, prec):
    """md_step replays its steps 2.. from captured CUDA graphs (blocks of 8); the
    result is bitwise that of the same stage schedule launched one md_stage at a
    time, for both ping-pong parities (odd step counts alternate them between
    calls).  md_step launches no more kernels than the stage-by-stage run (its
    first stage reuses the cached force of the previous call)."""
    from paper_1212_0262_gb300.system import stage_schedule

    N = 3000
    a, _, _ = _sys(model, N, prec)
    b, _, _ = _sys(model, N, prec)
    la, lb = a.launch_count, b.launch_count
    for n in (17, 17, 9, 25, 1):
        a.step(n)
        for bb, dd in stage_schedule(n):
            b.stage(bb, dd)
        qa, pa = a.get_state()
        qb, pb = b.get_state()
        assert np.array_equal(qa, qb) and np.array_equal(pa, pb), n
    assert a.launch_count - la <= b.launch_count - lb


@pytest.mark.parametrize("model", [0, 1, 2])
def test_step_on_the_legacy_default_stream(model):
    """The legacy default stream cannot be captured: md_step then launches every
    stage itself, with the same result."""
    a, _, _ = _sys(model, 2000, "mixed")
    b, _, _ = _sys(model, 2000, "mixed")
    b.set_stream(0)
    a.step(20)
    b.step(20)
    qa, pa = a.get_state()
    qb, pb = b.get_state()
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)


@pytest.mark.parametrize("offset", [1e3, -2.5e4, 3e6])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
@pytest.mark.parametrize("model", [0, 1])
def test_large_angles_keep_parity(model, prec, tol, offset):
    """The FP64 state is never wrapped, so angles grow over long runs; the FP32 paths
    reduce theta - 2 pi k before FP32 arithmetic (HMF: float-pair split and FP32
    Cody-Waite; Ring mirror: FP64 Cody-Waite).  Forces at angles shifted far from
    [-pi, pi) keep the bounds."""
    N = 2049
    q, p = inputs.default_state(model, N, 77)
    q = q + offset
    with System(model, N, EPS[model], 0.05, 1, precision=prec) as s:
        s.set_state(q, p)
        f = s.force()
    fo = ora.force(model, q, EPS[model])
    scale = ora.force_abs(model, q, EPS[model])
    # the angles themselves carry |theta| ulp(1) of representation error in FP64
    slack = 0.0 if prec == "mixed" else 4 * abs(offset) * 2.2e-16 * scale
    assert np.all(np.abs(f - fo) <= tol * scale + slack + 1e-300), (np.abs(f - fo) / scale).max()


def test_small_config_hmf_n1e4_fp64_100_steps():
    """The small configuration as stated: HMF, N = 10,000, FP64, water-bag theta in
    [-1, 1), p in [-1.2, 1.2) (seed 1), dt = 0.1, 100 steps; total energy,
    magnetization and relative energy error against the oracle's run of the same
    steps (mean-field HMF has a small Lyapunov exponent, so summation-order
    differences stay near rounding over this span)."""
    N, dt, nsteps = 10_000, 0.1, 100
    q0, p0 = inputs.waterbag(N, 1)
    with System(0, N, 0.0, dt, 1, precision="fp64") as s:
        s.set_state(q0, p0)
        e0 = sum(s.energy())
        s.step(nsteps)
        q, p = s.get_state()
        K, V = s.energy()
        mx, my = s.magnetization()
    qo, po = ora.step(0, q0, p0, 0.0, dt, nsteps)
    assert np.max(np.abs(q - qo)) <= 1e-10 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-10 * max(1.0, np.abs(po).max())
    eo = ora.energy(0, qo, po)
    e0o = ora.energy(0, q0, p0)
    assert abs((K + V) - eo) <= 1e-10 * abs(eo)
    assert abs(e0 - e0o) <= 1e-12 * abs(e0o)
    mxo, myo = ora.magnetization(qo)
    assert abs(mx - mxo) < 1e-10 and abs(my - myo) < 1e-10
    de, deo = abs((K + V - e0) / e0), abs((eo - e0o) / e0o)
    assert abs(de - deo) <= 1e-3 * deo + 1e-13, (de, deo)


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4])
def test_switching_precision_eps_and_state_between_steps(model):
    """Every cache (force, mirrors in both record formats, HMF sums and the FP64
    (cos, sin) buffer, step graphs) follows precision switches, eps changes and
    state replacements between steps: the run matches the oracle's run of the same
    segments (FP32 pair arithmetic in the mixed segments bounds the agreement)."""
    eps = {0: 0.0, 1: 0.01, 2: 1e-3, 3: 1e-3, 4: 1e-3}[model]
    eps2 = {0: 0.0, 1: 0.02, 2: 2e-3, 3: 2e-3, 4: 0.0}[model]
    N, dt = 1000, 0.02
    q0, p0 = inputs.default_state(model, N, 90)
    with System(model, N, eps, dt, 1, precision="fp64") as s:
        s.set_state(q0, p0)
        s.step(3)
        s.set_precision("mixed")
        s.step(10)
        s.set_precision("fp64")
        s.step(9)
        s.set_eps(eps2)
        s.step(3)
        qm, pm = s.get_state()
        q1, p1 = inputs.default_state(model, N, 91)
        s.set_state(q1, p1)
        s.step(2)
        q, p = s.get_state()
    qo, po = ora.step(model, q0, p0, eps, dt, 22)
    qo, po = ora.step(model, qo, po, eps2, dt, 3)
    assert np.max(np.abs(qm - qo)) <= 1e-5 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(pm - po)) <= 1e-5 * max(1.0, np.abs(po).max())
    qo, po = ora.step(model, q1, p1, eps2, dt, 2)
    assert np.max(np.abs(q - qo)) <= 1e-11 * max(1.0, np.abs(qo).max())
    assert np.max(np.abs(p - po)) <= 1e-11 * max(1.0, np.abs(po).max())

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
identities (Eq. 2 pair sum vs the mean-field Eqs. 5-7), the definition of a
force as minus the gradient of the Hamiltonians of Eqs. 1-3 (central finite
differences), the order and time reversibility of the Eq. 4 splitting (exact
harmonic-oscillator flow, Delta t^4 energy-error slope), conservation laws that
follow from pair antisymmetry, special cases with known answers, and finite
differences of the discrete adjoint.
"""
import math
import os

import numpy as np
import pytest

from paper_1212_0262_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state(model, N, seed):
    if model == 0:
        return inputs.waterbag(N, seed)
    if model == 1:
        return inputs.ring_state(N, seed)
    if model == 3:
        return inputs.ball_state(N, seed)
    if model == 4:
        return inputs.sheet_state(N, seed)
    return inputs.disk_state(N, seed)


# ------------------------------------------------------------ Eq. 4 -------

def test_yoshida_matches_published_weights(ora):
    B0, B1, D0, D1 = ora.yoshida()
    vals = {}
    with open(os.path.join(GOLDEN, "yoshida_coefficients.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert abs(D0 - vals["w1"]) < 1e-14
    assert abs(D1 - vals["w0"]) < 1e-14
    assert abs(B0 - vals["w1"] / 2) < 1e-14
    assert abs(B1 - (vals["w0"] + vals["w1"]) / 2) < 1e-14


def test_yoshida_consistency_and_order_conditions(ora):
    B0, B1, D0, D1 = ora.yoshida()
    assert abs(2 * B0 + 2 * B1 - 1.0) < 1e-15      # kicks sum to one step
    assert abs(2 * D0 + D1 - 1.0) < 1e-15          # drifts sum to one step
    assert abs(2 * D0 ** 3 + D1 ** 3) < 1e-14      # third-order error cancels


def test_harmonic_local_error_is_fifth_order(ora):
    """One step of the oracle on q'' = -q against the exact rotation: the local
    error is O(dt^5), so halving dt divides it by 32."""
    q0, p0 = np.array([1.0]), np.array([0.3])
    errs = []
    for h in (0.2, 0.1, 0.05):
        q, p = ora.step(ora.HARMONIC, q0, p0, 0.0, h, 1)
        qe = q0[0] * math.cos(h) + p0[0] * math.sin(h)
        pe = -q0[0] * math.sin(h) + p0[0] * math.cos(h)
        errs.append(math.hypot(q[0] - qe, p[0] - pe))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 28 < r1 < 36 and 28 < r2 < 36, (errs, r1, r2)


def test_harmonic_global_error_is_fourth_order(ora):
    q0, p0 = np.array([1.0]), np.array([0.0])
    errs = []
    for n in (20, 40, 80):
        q, p = ora.step(ora.HARMONIC, q0, p0, 0.0, 4.0 / n, n)
        errs.append(abs(q[0] - math.cos(4.0)) + abs(p[0] + math.sin(4.0)))
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18, errs


def test_energy_error_slope_is_four_hmf_waterbag(ora):
    """Max |E(t) - E0| over a fixed time window scales as dt^4 (HMF water-bag)."""
    q0, p0 = inputs.waterbag(500, 11)
    e0 = ora.energy(ora.HMF, q0, p0)
    T = 3.2
    dts = [0.2, 0.1, 0.05, 0.025]
    errs = []
    for dt in dts:
        q, p = q0.copy(), p0.copy()
        worst = 0.0
        for _ in range(int(round(T / dt))):
            q, p = ora.step(ora.HMF, q, p, 0.0, dt, 1)
            worst = max(worst, abs(ora.energy(ora.HMF, q, p) - e0))
        errs.append(worst)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 3.7 < slope < 4.3, (errs, slope)


def test_time_reversibility(ora):
    """n steps, negate p, n steps, negate p: back to the start (Sec. 3, Eq. 4)."""
    for model, eps in ((0, 0.0), (1, 0.01), (2, 1e-3)):
        q0, p0 = _state(model, 32, 5 + model)
        q, p = ora.step(model, q0, p0, eps, 0.02, 10)
        q, p = ora.step(model, q, -p, eps, 0.02, 10)
        assert np.max(np.abs(q - q0)) < 1e-12
        assert np.max(np.abs(-p - p0)) < 1e-12


# ------------------------------------------------- models (Eqs. 1-3, 5-7) --

@pytest.mark.parametrize("N", [1, 2, 7, 64])
def test_hmf_meanfield_equals_pairwise(ora, N):
    q, _ = inputs.waterbag(N, 100 + N, -3.0, 3.0)
    f_mf = ora.force(ora.HMF, q)
    f_pw = ora.force_hmf_pairwise(q)
    scale = ora.force_abs(ora.HMF, q) + 1e-300
    assert np.max(np.abs(f_mf - f_pw) / np.maximum(scale, 1.0 / N)) < 1e-13
    v_mf = ora.potential(ora.HMF, q)
    v_pw = ora.potential_hmf_pairwise(q)
    assert abs(v_mf - v_pw) <= 1e-13 * max(1.0, N)


@pytest.mark.parametrize("N,alpha", [(1, 0.3), (1001, 2.5e-3), (4096, 1.7e-3), (50_000, 1e-4)])
def test_hmf_closed_form_magnetization_of_an_arithmetic_progression(ora, N, alpha):
    """Eq. 7 for theta_i = alpha i: the geometric sum of e^{i alpha k} gives
    M = e^{i alpha (N-1)/2} sin(alpha N/2) / (N sin(alpha/2)); the mean-field force of
    Eq. 6 is then f_i = cos(theta_i) My - sin(theta_i) Mx (sign: particles are pulled
    towards the direction of M).  The same closed form checks the GPU path at
    particle counts past 2^31."""
    q = alpha * np.arange(N, dtype=np.float64)
    amp = math.sin(alpha * N / 2) / (N * math.sin(alpha / 2))
    mx, my = math.cos(alpha * (N - 1) / 2) * amp, math.sin(alpha * (N - 1) / 2) * amp
    ox, oy = ora.magnetization(q)
    assert abs(ox - mx) < 1e-14 and abs(oy - my) < 1e-14
    f = ora.force(ora.HMF, q)
    assert np.max(np.abs(f - (np.cos(q) * my - np.sin(q) * mx))) < 1e-14
    # towards M: a particle a quarter turn behind M is pulled forward
    phi = math.atan2(my, mx)
    assert ora.force(ora.HMF, np.append(q, phi - math.pi / 2))[-1] > 0


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (1, 1.0), (2, 1e-3), (2, 0.5), (3, 1e-3), (3, 0.5),
                                       (4, 1e-3), (4, 0.5)])
def test_force_is_minus_gradient_of_potential(ora, model, eps):
    N = 12
    q, _ = _state(model, N, 21)
    f = ora.force(model, q, eps)
    h = 1e-5
    fd = np.empty_like(q)
    for k in range(q.size):
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        fd[k] = -(ora.potential(model, qp, eps) - ora.potential(model, qm, eps)) / (2 * h)
    scale = np.max(np.abs(f))
    assert np.max(np.abs(fd - f)) < 2e-7 * scale, np.max(np.abs(fd - f)) / scale


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (2, 1e-3), (3, 1e-3), (4, 0.0), (4, 1e-3)])
def test_total_momentum_conserved(ora, model, eps):
    N = 40
    q0, p0 = _state(model, N, 31)
    q, p = ora.step(model, q0, p0, eps, 0.05, 20)
    d = {2: 2, 3: 3}.get(model, 1)
    for c in range(d):
        tot0 = p0[c * N:(c + 1) * N].sum()
        tot = p[c * N:(c + 1) * N].sum()
        assert abs(tot - tot0) < 1e-13 * np.abs(p0).sum() * 20


def test_angular_momentum_conserved_2d(ora):
    N = 40
    q0, p0 = inputs.disk_state(N, 41)
    q, p = ora.step(2, q0, p0, 1e-3, 0.05, 20)

    def lz(q, p):
        return np.sum(q[:N] * p[N:] - q[N:] * p[:N])

    assert abs(lz(q, p) - lz(q0, p0)) < 1e-12 * np.sum(np.abs(q0) * np.abs(p0).max()) * 20


def test_angular_momentum_conserved_3d(ora):
    N = 40
    q0, p0 = inputs.ball_state(N, 43)

    def L(q, p):
        r, v = q.reshape(3, N).T, p.reshape(3, N).T
        return np.cross(r, v).sum(axis=0)

    q, p = ora.step(3, q0, p0, 1e-3, 0.05, 20)
    scale = np.sum(np.abs(q0)) * np.abs(p0).max()
    assert np.max(np.abs(L(q, p) - L(q0, p0))) < 1e-12 * scale * 20


def test_sheet_force_is_a_count_of_neighbours_on_each_side(ora):
    """eps = 0: f_i = (number of sheets to the right - number to the left) / N,
    counted here by sorting (independent of the oracle's pair loop); exact."""
    N = 301
    x, _ = inputs.sheet_state(N, 61)
    x[5] = x[9]  # a coincident pair: sign(0) = 0
    srt = np.sort(x)
    left = np.searchsorted(srt, x, side="left")
    right = N - np.searchsorted(srt, x, side="right")
    expect = (right - left) / N
    f = ora.force(4, x, 0.0)
    assert np.array_equal(f, expect)
    assert f.sum() == 0.0


def test_sheet_force_is_minus_gradient_of_piecewise_linear_potential(ora):
    """eps = 0: V is linear between crossings, so central differences with a step
    below the smallest gap are exact up to rounding."""
    N = 40
    x = np.sort(inputs.uniform(62, 0, N)) * 2 - 1
    h = 0.25 * np.min(np.diff(x))
    f = ora.force(4, x, 0.0)
    for k in range(N):
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd = -(ora.potential(4, xp, 0.0) - ora.potential(4, xm, 0.0)) / (2 * h)
        assert abs(fd - f[k]) < 1e-9


def test_sheet_pair_bounce_period(ora):
    """Two sheets released at separation u0: the separation obeys u'' = -sign(u)
    (coupling 1/N with N = 2), so they cross and return after T = 4 sqrt(2 u0).  The
    force jumps at the crossing, so the return error falls only linearly with dt."""
    u0 = 0.5
    T = 4 * math.sqrt(2 * u0)
    q0, p0 = np.array([u0 / 2, -u0 / 2]), np.zeros(2)
    errs = []
    for n in (400, 800):
        q, p = ora.step(4, q0, p0, 0.0, T / n, n)
        errs.append(np.max(np.abs(q - q0)))
        assert np.max(np.abs(q - q0)) < 4.0 / n and np.max(np.abs(p - p0)) < 8.0 / n
    assert 1.6 < errs[0] / errs[1] < 2.4


def test_sheet_fp32_decisions(ora):
    """The FP32-decision force equals the FP64 one when the FP32 roundings keep every
    order, and counts an FP32 tie as 0."""
    x = np.linspace(-1, 1, 257)
    assert np.array_equal(ora.force_sheet_f32(x), ora.force(4, x, 0.0))
    y = np.array([0.5, 0.5 + 1e-12, -0.25])  # distinct in FP64, equal in FP32
    f64, f32 = ora.force(4, y, 0.0), ora.force_sheet_f32(y)
    assert f64[0] == -(-1 + 1) / 3 + 0.0 and f64[1] == -(1 + 1) / 3
    assert f32[0] == f32[1] == -1 / 3


def test_3d_shell_theorem(ora):
    """Newton's shell theorem: 12 unit masses on the vertices of an icosahedron of
    radius a (a spherical 5-design: its multipole moments of orders 1 to 5 vanish)
    act on a distant test mass like 12 masses at the centre, up to O((a/D)^6)."""
    phi = (1 + math.sqrt(5)) / 2
    verts = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            verts += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    v = np.array(verts, dtype=float)
    a, D = 0.05, 1.0
    v *= a / np.linalg.norm(v[0])
    test = np.array([[0.6, -0.48, 0.64]]) * D  # |test| = D, a generic direction
    r = np.vstack([v, test])
    N = r.shape[0]
    q = r.T.reshape(-1)
    f = ora.force(3, q, 0.0).reshape(3, N)[:, -1]
    f_point = -(12.0 / N) * test[0] / D ** 3
    assert np.max(np.abs(f - f_point)) < 1e-6 * np.linalg.norm(f_point)
    # and the potential energy of the test mass, to the same order
    V_all = ora.potential(3, q, 0.0)
    V_shell = ora.potential(3, v.T.reshape(-1), 0.0) * 12 / N  # same 1/N coupling
    assert abs((V_all - V_shell) - (-12.0 / (N * D))) < 1e-6 * 12.0 / (N * D)


def test_ring_is_3d_gravity_on_the_unit_circle(ora):
    """The Ring model (Eq. 1) is softened 3D gravity restricted to the unit circle:
    |r_i - r_j|^2 = 2 (1 - cos(theta_i - theta_j)), so with the 3D softening 2 eps
    V_ring(theta, eps) = V_3D((cos, sin, 0), 2 eps), and the Ring force is the
    tangential component (-sin, cos, 0) . F_3D of the 3D force (chord geometry, not
    the Ring formulas: a wrong sqrt(2), eps or sign in either fails)."""
    rng = np.random.default_rng(12)
    N, eps = 37, 0.01
    th = rng.uniform(-np.pi, np.pi, N) + 2 * np.pi * rng.integers(-3, 4, N)
    q3 = np.concatenate([np.cos(th), np.sin(th), np.zeros(N)])
    v_r, v_3 = ora.potential(1, th, eps), ora.potential(3, q3, 2 * eps)
    assert abs(v_r - v_3) <= 1e-13 * abs(v_r)
    F = ora.force(3, q3, 2 * eps).reshape(3, N)
    f_t = -np.sin(th) * F[0] + np.cos(th) * F[1]
    f_r = ora.force(1, th, eps)
    assert np.max(np.abs(f_r - f_t)) <= 1e-12 * np.max(ora.force_abs(1, th, eps))


def test_2d_shell_theorem_for_the_log_potential(ora):
    """Newton's theorem for the 2D (logarithmic) potential of Eq. 3: M unit masses on a
    regular M-gon of radius a act on a distant test mass like M masses at the centre,
    and exert no force on a mass inside, both up to O((ratio)^(M-1)); eps = 1e-12."""
    M, a, eps = 16, 0.05, 1e-12
    ang = 0.3 + 2 * np.pi * np.arange(M) / M
    ring = np.stack([a * np.cos(ang), a * np.sin(ang)], axis=1)
    D = 1.0
    test = np.array([0.6, -0.8]) * D
    r = np.vstack([ring, test])
    N = M + 1
    q = r.T.reshape(-1)
    f = ora.force(2, q, eps).reshape(2, N)[:, -1]
    f_point = -(2.0 / N) * M * test / D ** 2
    assert np.max(np.abs(f - f_point)) < 1e-9 * np.linalg.norm(f_point)
    V_all = ora.potential(2, q, eps)
    V_ring = ora.potential(2, ring.T.reshape(-1), eps) * M / N  # same 1/N coupling
    assert abs((V_all - V_ring) - (M / N) * math.log(D ** 2)) < 1e-9
    inside = np.vstack([ring / a * 0.1, [[0.012, 0.021]]])  # ring radius 0.1, |x| = 0.024
    fi = ora.force(2, inside.T.reshape(-1), eps).reshape(2, N)[:, -1]
    scale = (2.0 / N) * M / 0.1
    assert np.max(np.abs(fi)) < 1e-8 * scale


def test_3d_two_body_circular_orbit(ora):
    """Two unit masses at separation d with speeds v = 1/(2 sqrt(d)) (eps = 0, N = 2:
    coupling 1/2) move on a circle: the separation stays d and they are back at the
    start after one period 2 pi (d/2) / v."""
    d = 1.0
    v = 1.0 / (2.0 * math.sqrt(d))
    T = 2 * math.pi * (d / 2) / v
    q0 = np.array([d / 2, -d / 2, 0.0, 0.0, 0.0, 0.0])
    p0 = np.array([0.0, 0.0, v, -v, 0.0, 0.0])
    n = 800
    q, p = q0.copy(), p0.copy()
    for _ in range(4):
        q, p = ora.step(3, q, p, 0.0, T / n, n // 4)
        sep = np.linalg.norm(q.reshape(3, 2)[:, 0] - q.reshape(3, 2)[:, 1])
        assert abs(sep - d) < 2e-8
    err = np.max(np.abs(q - q0))
    assert err < 5e-8 and np.max(np.abs(p - p0)) < 5e-8
    # fourth order: halving the step divides the return error by about 16
    q2, _ = ora.step(3, q0, p0, 0.0, T / (n // 2), n // 2)
    assert 12.0 < np.max(np.abs(q2 - q0)) / err < 20.0


def test_special_cases(ora):
    # one HMF particle feels no force and drifts freely
    q, p = ora.step(ora.HMF, np.array([0.7]), np.array([0.25]), 0.0, 0.1, 10)
    assert ora.force(ora.HMF, np.array([0.7]))[0] == 0.0
    assert abs(q[0] - (0.7 + 10 * 0.1 * 0.25)) < 1e-14 and p[0] == 0.25
    # equally spaced angles: M = 0 and zero force (HMF and Ring, by symmetry)
    N = 64
    lat = 2 * np.pi * np.arange(N) / N - np.pi
    assert np.max(np.abs(ora.force(ora.HMF, lat))) < 1e-15
    fr = ora.force(ora.RING, lat, 0.01)
    assert np.max(np.abs(fr)) < 1e-13 * np.max(ora.force_abs(ora.RING, lat, 0.01))
    # two bodies: equal and opposite forces
    for model, eps, q in ((1, 0.01, np.array([0.3, -0.4])),
                          (2, 1e-3, np.array([0.1, -0.2, 0.05, 0.3])),
                          (3, 1e-3, np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.2]))):
        f = ora.force(model, q, eps)
        if model == 1:
            assert abs(f[0] + f[1]) < 1e-16
            assert f[0] < 0  # attraction: particle 0 sits at larger angle
        else:
            for c in range(model):
                assert abs(f[2 * c] + f[2 * c + 1]) < 1e-16
            assert f[0] < 0 and f[2] > 0  # pulled toward particle 1
    # one sheet, or sheets all at one place, feel no force
    assert ora.force(4, np.array([0.3]), 0.0)[0] == 0.0
    assert np.all(ora.force(4, np.full(5, 0.2), 0.0) == 0.0)
    # particles at rest have K = 0
    assert ora.kinetic(np.zeros(10)) == 0.0


def test_two_body_energy_conservation(ora):
    q0 = np.array([0.5, -0.5, 0.0, 0.0])
    p0 = np.array([0.0, 0.0, 0.4, -0.4])
    e0 = ora.energy(2, q0, p0, 1e-3)
    q, p = ora.step(2, q0, p0, 1e-3, 0.01, 200)
    assert abs(ora.energy(2, q, p, 1e-3) - e0) < 1e-7 * abs(e0)


# --------------------------------------------- derivatives and the adjoint -

@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (2, 1e-3), (3, 1e-3), (4, 1e-3), (4, 0.5)])
def test_hvp_matches_finite_difference_of_force(ora, model, eps):
    N = 16
    q, _ = _state(model, N, 51)
    v = inputs.uniform(52, 0, q.size) - 0.5
    jv = ora.hvp(model, q, v, eps)
    h = 1e-6
    fd = (ora.force(model, q + h * v, eps) - ora.force(model, q - h * v, eps)) / (2 * h)
    assert np.max(np.abs(jv - fd)) < 1e-7 * np.max(np.abs(jv))
    if model == 0:
        jmf = ora.hvp_hmf_meanfield(q, v)
        assert np.max(np.abs(jmf - jv)) < 1e-13 * np.max(np.abs(jv))


@pytest.mark.parametrize("model,eps", [(1, 0.01), (2, 1e-3), (3, 1e-3), (4, 1e-3), (4, 0.5)])
def test_dforce_deps_matches_finite_difference(ora, model, eps):
    q, _ = _state(model, 16, 61)
    h = 1e-7 * eps
    fd = (ora.force(model, q, eps + h) - ora.force(model, q, eps - h)) / (2 * h)
    de = ora.dforce_deps(model, q, eps)
    assert np.max(np.abs(de - fd)) < 1e-6 * np.max(np.abs(de))


@pytest.mark.parametrize("model,eps,obs", [(0, 0.0, 0), (0, 0.0, 1), (1, 0.01, 0), (1, 0.01, 1),
                                           (2, 1e-3, 0), (3, 1e-2, 0), (4, 0.05, 0)])
def test_adjoint_matches_central_differences(ora, model, eps, obs):
    N, dt, ns = 12, 0.05, 6
    q0, p0 = _state(model, N, 71 + model)
    val, gq, gp, ge = ora.grad(model, q0, p0, eps, dt, ns, obs)
    assert abs(val - ora.observable_after(model, q0, p0, eps, dt, ns, obs)) < 1e-14 * abs(val)
    h = 1e-6
    # every component
    for g, which in ((gq, 0), (gp, 1)):
        fd = np.empty_like(g)
        for k in range(g.size):
            a, b = q0.copy(), p0.copy()
            (a if which == 0 else b)[k] += h
            vp = ora.observable_after(model, a, b, eps, dt, ns, obs)
            (a if which == 0 else b)[k] -= 2 * h
            vm = ora.observable_after(model, a, b, eps, dt, ns, obs)
            fd[k] = (vp - vm) / (2 * h)
        assert np.max(np.abs(fd - g)) < 1e-6 * max(np.max(np.abs(g)), 1e-3), (which, fd, g)
    if model != 0:
        he = 1e-6 * eps
        fde = (ora.observable_after(model, q0, p0, eps + he, dt, ns, obs)
               - ora.observable_after(model, q0, p0, eps - he, dt, ns, obs)) / (2 * he)
        assert abs(fde - ge) < 1e-5 * max(abs(ge), 1e-6), (fde, ge)
    else:
        assert ge == 0.0


def test_step_matches_grad_forward_pass(ora):
    """The adjoint's forward pass re-evaluates f at every kick; its trajectory
    must be identical to the first-same-as-last step list."""
    q0, p0 = inputs.ring_state(20, 81)
    q, p = ora.step(1, q0, p0, 0.01, 0.05, 7)
    val, *_ = ora.grad(1, q0, p0, 0.01, 0.05, 7, 0)
    assert val == ora.kinetic(p)


def test_force_rows_equals_full_force_3d(ora):
    q, _ = inputs.ball_state(50, 71)
    full = ora.force(3, q, 1e-3).reshape(3, 50)
    rows = np.array([0, 7, 49])
    fr, ab = ora.force_rows(3, q, rows, 1e-3, with_abs=True)
    assert np.max(np.abs(fr - full[:, rows])) < 1e-15
    assert np.allclose(ab, ora.force_abs(3, q, 1e-3).reshape(3, 50)[:, rows], rtol=1e-14, atol=0)


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (2, 1e-3), (4, 0.0), (4, 1e-3)])
def test_force_rows_equals_full_force(ora, model, eps):
    q, _ = _state(model, 50, 91)
    rows = np.array([0, 7, 49, 23])
    full = ora.force(model, q, eps).reshape(2 if model == 2 else 1, 50)
    part, ab = ora.force_rows(model, q, rows, eps, with_abs=True)
    assert np.array_equal(full[:, rows], part)
    fa = ora.force_abs(model, q, eps).reshape(full.shape)
    np.testing.assert_allclose(ab, fa[:, rows], rtol=1e-14)

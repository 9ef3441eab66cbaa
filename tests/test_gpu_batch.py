"""Batched ensembles (md_batch_*) against the FP64 oracle, member by member.

Every system of an uneven ensemble, advanced in shared persistent launches and
replayed CUDA graphs, is compared element by element with the oracle: forces
(md_batch_force) within 1e-12 (FP64) or 2e-5 (mixed) of sum_j |f_ij| per particle
and component, and the state after 1 and 25 steps of the Sec. 3 step list (ora.step)
within the bounds that follow from those force bounds (see _traj_bounds).  Mixed
ensembles run the Newton's-third-law kernels by default (r = 0) and the one-sided
CUDA-core kernels with r = 4 or 8.  The comparisons with the same system advanced
alone by md_step (same pair arithmetic; only the stream-K split of the per-particle
sums differs) stay as extra checks."""
import functools

import numpy as np
import pytest

import oracle as ora
from paper_1212_0262_gb300 import Ensemble, System, inputs

pytestmark = pytest.mark.gpu

MODELS = [1, 2, 1, 2, 2, 1]
NS = [333, 1000, 2500, 4097, 777, 1500]
EPS = [0.01, 1e-3, 0.01, 1e-4, 1e-3, 0.05]
DTS = [0.05, 0.01, 0.05, 0.01, 0.01, 0.02]
SEEDS = [1000 + s for s in range(6)]


FORMS = {"mixed": ("mixed", None), "mixed_r4": ("mixed", 4), "mixed_r8": ("mixed", 8), "fp64": ("fp64", None)}


def _ensemble(form):
    """The uneven ensemble in `form`, every member set to the host generator's state
    (the oracle's starting point, bit for bit)."""
    prec, r = FORMS[form]
    ens = Ensemble(MODELS, NS, EPS, DTS, SEEDS, precision=prec)
    if r is not None:
        ens.set_tuning(r, 0.5, 0)
    for s in range(len(NS)):
        ens.set_state(s, *inputs.default_state(MODELS[s], NS[s], SEEDS[s]))
    return ens


@functools.lru_cache(maxsize=None)
def _oracle_run(s, nsteps):
    q0, p0 = inputs.default_state(MODELS[s], NS[s], SEEDS[s])
    q, p = ora.step(MODELS[s], q0, p0, EPS[s], DTS[s], nsteps)
    return q0, p0, q, p, float(ora.force_abs(MODELS[s], q0, EPS[s]).max())


def _traj_bounds(s, nsteps, prec, q, p, fscale):
    """Bounds on |q - q_ora| and |p - p_ora| after nsteps.  FP64: the summation-order
    bounds of the single-system tests (1e-12 after one step, 1e-11 after 25).  Mixed:
    each kick's force is within 2e-5 sum_j |f_ij| of the FP64 one, so one step moves p
    by at most sum|b| dt 2e-5 S from the oracle (S the largest scale), n steps by n
    times that, and q by the drifts of those errors, sum|d| dt per step summed over
    the steps; a factor 4 covers the growth of differences along the trajectory
    (t <= 1.25 here) and 1e-12 the FP64 state arithmetic."""
    B0, B1, D0, D1 = ora.yoshida()
    sb, sd = 2 * abs(B0) + 2 * abs(B1), 2 * abs(D0) + abs(D1)
    dt = DTS[s]
    if prec == "fp64":
        t = 1e-12 if nsteps == 1 else 1e-11
        return t * max(1.0, np.abs(q).max()), t * (np.abs(p).max() + dt * fscale)
    dp1 = sb * dt * 2e-5 * 1.1 * fscale
    G = 4.0
    bp = G * nsteps * dp1 + 1e-12 * np.abs(p).max()
    bq = G * sd * dt * dp1 * nsteps * (nsteps + 1) / 2 + 1e-12 * max(1.0, np.abs(q).max())
    return bq, bp


@pytest.mark.parametrize("form", list(FORMS))
def test_ensemble_forces_match_the_oracle(form):
    """md_batch_force of every member against ora.force, element by element."""
    ens = _ensemble(form)
    f = ens.force()
    tol = 1e-12 if form == "fp64" else 2e-5
    for s in range(len(NS)):
        q, _ = ens.get_state(s)
        fo = ora.force(MODELS[s], q, EPS[s])
        scale = ora.force_abs(MODELS[s], q, EPS[s])
        err = np.abs(f[s] - fo)
        assert np.all(err <= tol * scale + 1e-300), (s, (err / np.maximum(scale, 1e-300)).max())
    ens.close()


@pytest.mark.parametrize("form", ["fp64", "mixed", "mixed_r8"])
@pytest.mark.parametrize("nsteps", [1, 25])
def test_ensemble_trajectories_match_the_oracle(form, nsteps):
    """Every member after 1 and 25 steps (25: the first step, two replays of the
    10-step graph and four launched steps) against ora.step from the same state."""
    ens = _ensemble(form)
    ens.step(nsteps)
    for s in range(len(NS)):
        q0, p0, qo, po, fscale = _oracle_run(s, nsteps)
        q, p = ens.get_state(s)
        bq, bp = _traj_bounds(s, nsteps, FORMS[form][0], qo, po, fscale)
        assert np.max(np.abs(q - qo)) <= bq, (s, np.max(np.abs(q - qo)), bq)
        assert np.max(np.abs(p - po)) <= bp, (s, np.max(np.abs(p - po)), bp)
    ens.close()


def _one_sided(sy):
    # the one-sided batched kernel is the one-sided CUDA-core kernel of the single-system path
    sy.set_tuning("ring_tc", 0)
    sy.set_tuning("symmetric", 0)
    return sy


def _alone(s, nsteps, prec, sym=False):
    with System(MODELS[s], NS[s], EPS[s], DTS[s], SEEDS[s], precision=prec) as sy:
        (sy if sym else _one_sided(sy)).step(nsteps)
        return sy.get_state(), sy.energy()


@pytest.mark.parametrize("prec", ["mixed", "mixed_one_sided", "fp64"])
@pytest.mark.parametrize("nsteps", [1, 25])
def test_ensemble_matches_individual_runs(prec, nsteps):
    ens = Ensemble(MODELS, NS, EPS, DTS, SEEDS, precision=prec.split("_")[0])
    if prec == "mixed_one_sided":
        ens.set_tuning(8, 0.5, 0)
    ens.step(nsteps)
    K, V = ens.energy()
    for s in range(len(NS)):
        (q, p), (k, v) = _alone(s, nsteps, prec.split("_")[0], sym=(prec == "mixed"))
        qb, pb = ens.get_state(s)
        tol = 1e-12 if prec == "fp64" else 1e-9
        assert np.max(np.abs(qb - q)) <= tol * max(1.0, np.abs(q).max()), s
        assert np.max(np.abs(pb - p)) <= tol * max(1.0, np.abs(p).max()), s
        assert abs(K[s] - k) <= 1e-9 * abs(k) and abs(V[s] - v) <= 1e-9 * max(abs(v), 1.0)
    ens.close()


def test_autotune_leaves_states_unchanged_and_shapes_agree():
    ens = Ensemble(MODELS, NS, EPS, DTS, SEEDS)
    before = [ens.get_state(s) for s in range(len(NS))]
    best = ens.autotune()
    assert best > 0.0
    for s in range(len(NS)):
        q, p = ens.get_state(s)
        assert np.array_equal(q, before[s][0]) and np.array_equal(p, before[s][1])
    ens.step(12)
    ref = [ens.get_state(s) for s in range(len(NS))]
    r = ens.tuning[0]  # the form autotune picked; other splits and CTA counts must agree with it
    for split, cps in ((0.3, 0), (0.7, 2)):
        e2 = Ensemble(MODELS, NS, EPS, DTS, SEEDS)
        e2.set_tuning(r, split, cps)
        e2.step(12)
        for s in range(len(NS)):
            q, p = e2.get_state(s)
            assert np.max(np.abs(q - ref[s][0])) <= 1e-9 * max(1.0, np.abs(q).max())
        e2.close()
    ens.close()


def test_set_state_is_used_by_the_next_step():
    ens = Ensemble(MODELS[:2], NS[:2], EPS[:2], DTS[:2], SEEDS[:2])
    q, p = inputs.default_state(MODELS[1], NS[1], 5)
    ens.set_state(1, q, p)
    ens.step(3)
    with System(MODELS[1], NS[1], EPS[1], DTS[1], 0, precision="mixed") as sy:
        sy.set_state(q, p)
        sy.step(3)
        qa, pa = sy.get_state()
    qb, pb = ens.get_state(1)
    assert np.max(np.abs(qb - qa)) <= 1e-9 * max(1.0, np.abs(qa).max())
    ens.close()


def test_one_sided_tunings_agree_with_the_symmetric_default():
    """r = 4 and r = 8 (one-sided) and r = 0 (symmetric) give the same trajectories
    to the FP32 pair-arithmetic level."""
    ref = Ensemble(MODELS, NS, EPS, DTS, SEEDS)
    ref.step(5)
    for r in (4, 8):
        e2 = Ensemble(MODELS, NS, EPS, DTS, SEEDS)
        e2.set_tuning(r, 0.5, 0)
        e2.step(5)
        for s in range(len(NS)):
            q, p = e2.get_state(s)
            qr, pr = ref.get_state(s)
            assert np.max(np.abs(q - qr)) <= 1e-5 * max(1.0, np.abs(qr).max()), (r, s)
        e2.close()
    ref.close()


def test_bench_ensemble_sampled_forces_match_the_oracle():
    """The 256-system ensemble of the bench (128 Ring at eps = 0.01, 128 2D at
    eps = 1e-4, N = floor(4096 16^u)), autotuned as the bench runs it: the forces of
    the smallest and largest system of each model, on 64 sampled particles (the first
    and last included), within 2e-5 sum_j |f_ij| of ora.force_rows."""
    nsys = 256
    Ns = inputs.ensemble_sizes(nsys, 1000)
    models = [1 if s < nsys // 2 else 2 for s in range(nsys)]
    eps = [0.01 if m == 1 else 1e-4 for m in models]
    dts = [0.05 if m == 1 else 0.01 for m in models]
    seeds = [1000 + s for s in range(nsys)]
    ens = Ensemble(models, Ns, eps, dts, seeds, precision="mixed")
    ens.autotune()
    half = nsys // 2
    pick = [int(np.argmin(Ns[:half])), int(np.argmax(Ns[:half])),
            half + int(np.argmin(Ns[half:])), half + int(np.argmax(Ns[half:]))]
    f = ens.force(pick)
    rng = np.random.default_rng(5)
    for s in pick:
        N = int(Ns[s])
        rows = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 62)]))
        q, _ = ens.get_state(s)
        fo, scale = ora.force_rows(models[s], q, rows, eps[s], with_abs=True)
        fg = f[s].reshape(-1, N)[:, rows]
        err = np.abs(fg - fo)
        assert np.all(err <= 2e-5 * scale + 1e-300), (s, (err / np.maximum(scale, 1e-300)).max())
    ens.close()


def test_bench_ensemble_sampled_systems_match_the_single_system_path():
    """The 256-system ensemble of the bench (128 Ring at eps = 0.01, 128 2D at
    eps = 1e-4, N = floor(4096 16^u)), autotuned as the bench runs it: after one
    step, the smallest and largest system of each model equal the same system
    advanced alone by md_step (whose forces the full-size sampled parity tests pin to
    the oracle) to rounding; after two steps every system's energy error is within
    twice that of the same ensemble run in FP64."""
    nsys = 256
    Ns = inputs.ensemble_sizes(nsys, 1000)
    models = [1 if s < nsys // 2 else 2 for s in range(nsys)]
    eps = [0.01 if m == 1 else 1e-4 for m in models]
    dts = [0.05 if m == 1 else 0.01 for m in models]
    seeds = [1000 + s for s in range(nsys)]
    ens = Ensemble(models, Ns, eps, dts, seeds, precision="mixed")
    ens.autotune()
    K0, V0 = ens.energy()
    ens.step(1)
    half = nsys // 2
    pick = [int(np.argmin(Ns[:half])), int(np.argmax(Ns[:half])),
            half + int(np.argmin(Ns[half:])), half + int(np.argmax(Ns[half:]))]
    for s in pick:
        with System(models[s], int(Ns[s]), eps[s], dts[s], seeds[s], precision="mixed") as sy:
            sy.step(1)
            q, p = sy.get_state()
        qb, pb = ens.get_state(s)
        assert np.max(np.abs(qb - q)) <= 1e-9 * max(1.0, np.abs(q).max()), s
        assert np.max(np.abs(pb - p)) <= 1e-9 * max(1.0, np.abs(p).max()), s
    ens.step(1)
    K, V = ens.energy()
    e0 = K0 + V0
    de_mixed = np.abs(K + V - e0) / np.abs(e0)
    ens.close()
    ref = Ensemble(models, Ns, eps, dts, seeds, precision="fp64")
    Kr0, Vr0 = ref.energy()
    assert np.allclose(Kr0 + Vr0, e0, rtol=1e-12, atol=0.0)
    ref.step(2)
    Kr, Vr = ref.energy()
    de_fp64 = np.abs(Kr + Vr - e0) / np.abs(e0)
    ref.close()
    assert np.all(de_mixed <= 2.0 * de_fp64 + 1e-9), np.max(de_mixed - 2.0 * de_fp64)

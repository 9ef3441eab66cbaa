"""The seeded input generator: SplitMix64 known-answer values and the shape of
each initial-state recipe."""
import os

import numpy as np

from paper_1212_0262_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_known_answers():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert rows
    for seed, *outs in rows:
        got = inputs.splitmix64(int(seed), np.arange(3))
        assert [int(x) for x in got] == [int(o) for o in outs]


def test_uniform_range_and_moments():
    u = inputs.uniform(3, 0, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.002


def test_gaussian_moments():
    g = inputs.gaussian(4, 0, 200000)
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 0.02


def test_recipes():
    q, p = inputs.waterbag(1000, 1)
    assert q.min() >= -1.0 and q.max() < 1.0 and p.min() >= -1.2 and p.max() < 1.2
    q, p = inputs.ring_state(1000, 3)
    assert q.min() >= -np.pi and q.max() < np.pi and abs(p.std() - 0.5) < 0.05
    q, p = inputs.disk_state(1000, 4)
    r = np.hypot(q[:1000], q[1000:])
    assert r.max() <= 1.0 and q.size == 2000 and p.size == 2000
    q, p = inputs.annulus_state(1000, 5)
    r = np.hypot(q[:1000], q[1000:])
    assert r.min() >= 1.0 - 1e-15 and r.max() < 1.5 and not p.any()
    n = inputs.ensemble_sizes(256, 1000)
    assert n.min() >= 4096 and n.max() < 65536


def test_counter_based_draws_are_prefix_stable():
    a = inputs.uniform(9, 0, 100)
    b = inputs.uniform(9, 40, 20)
    assert np.array_equal(a[40:60], b)


def test_ball_state_recipe():
    """3D ball: deterministic, inside the unit ball, uniform in volume (mean r^3 = 1/2,
    mean z = 0), counters 3i..3i+2 per particle, then Gaussian momenta."""
    q, p = inputs.ball_state(20000, 5)
    q2, p2 = inputs.ball_state(20000, 5)
    assert np.array_equal(q, q2) and np.array_equal(p, p2)
    r = np.sqrt(q[:20000] ** 2 + q[20000:40000] ** 2 + q[40000:] ** 2)
    assert r.max() <= 1.0 + 1e-15
    assert abs(np.mean(r ** 3) - 0.5) < 0.01
    assert abs(np.mean(q[40000:])) < 0.01
    u = inputs.uniform(5, 0, 3)
    assert abs(r[0] - np.cbrt(u[0])) < 1e-15 and abs(q[40000] - np.cbrt(u[0]) * (1 - 2 * u[1])) < 1e-15
    assert abs(np.std(p) - 0.3) < 0.01
    q3, p3 = inputs.default_state(3, 10, 2)
    assert q3.size == 30 and p3.size == 30


def test_sheet_state_recipe():
    """1D sheets: the water-bag counters and maps with x in [-1, 1), p in [-0.5, 0.5)."""
    q, p = inputs.sheet_state(1000, 9)
    qw, pw = inputs.waterbag(1000, 9, -1.0, 1.0, -0.5, 0.5)
    assert np.array_equal(q, qw) and np.array_equal(p, pw)
    assert q.min() >= -1.0 and q.max() < 1.0 and p.min() >= -0.5 and p.max() < 0.5
    q4, p4 = inputs.default_state(4, 1000, 9)
    assert np.array_equal(q4, q)

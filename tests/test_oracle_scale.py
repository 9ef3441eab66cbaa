"""Pins of the oracle's force scale, sum_j |f_ij| (ora_force_abs and the out_abs of
ora_force_rows), from the mathematics rather than from a second copy of its formula.

Every GPU parity bound is tol * sum_j |f_ij|, so a wrong factor in the scale would
loosen (or tighten) all of them at once.  Two facts fix it:
  * the triangle inequality, |f_i| = |sum_j f_ij| <= sum_j |f_ij|, on any state;
  * equality when every pair term acting on particle i has the same sign: the end
    particle of a collinear set (2D, 3D: all coordinate differences of one sign),
    the outermost sheet, a Ring particle with all others within (0, pi) ahead of it,
    and for HMF's mean-field terms cos(th_i) My and sin(th_i) Mx a particle at
    th_i = 0 (or pi/2) with all others where sin (or cos) is positive.
The last test plants factor and index mistakes in copies of the oracle (compiled
here, on the CPU) and checks that these pins catch each one.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1212_0262_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "md_oracle.c")


class Api:
    """force / force_abs / force_rows over one build of the oracle C source."""

    def __init__(self, lib):
        P = ctypes.POINTER(ctypes.c_double)
        lib.ora_force.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, P, P]
        lib.ora_force_abs.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, P, P]
        lib.ora_force_rows.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, P,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, P, P]
        self.lib = lib

    @staticmethod
    def _p(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def force(self, model, q, eps):
        q = np.ascontiguousarray(q, dtype=np.float64)
        f = np.empty_like(q)
        self.lib.ora_force(model, q.size // _dim(model), eps, self._p(q), self._p(f))
        return f

    def force_abs(self, model, q, eps):
        q = np.ascontiguousarray(q, dtype=np.float64)
        a = np.empty_like(q)
        self.lib.ora_force_abs(model, q.size // _dim(model), eps, self._p(q), self._p(a))
        return a

    def rows_abs(self, model, q, rows, eps):
        q = np.ascontiguousarray(q, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(_dim(model) * rows.size)
        ab = np.empty_like(out)
        self.lib.ora_force_rows(model, q.size // _dim(model), eps, self._p(q),
                                rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size,
                                self._p(out), self._p(ab))
        return out.reshape(_dim(model), rows.size), ab.reshape(_dim(model), rows.size)


def _dim(model):
    return 2 if model == 2 else 3 if model == 3 else 1


@pytest.fixture(scope="module")
def api(ora):
    return Api(ora._load())


# ------------------------------------------------------------ states -------

def _collinear(N, dim, seed):
    """N distinct points on a line through the origin with direction of all-positive
    components, sorted by the parameter: particle N-1 has every coordinate difference
    to the others positive, particle 0 every one negative."""
    t = np.sort(inputs.uniform(seed, 0, N) * 2.0 - 1.0)
    u = np.array([1.0, 2.0, 3.0][:dim])
    u /= np.linalg.norm(u)
    return np.concatenate([t * u[c] for c in range(dim)])


def _same_sign_cases():
    """(model, eps, q, rows) with every pair term on each listed row of one sign."""
    N = 57
    cases = []
    for eps in (1e-3, 0.0):  # 2D and 3D at eps = 0 are never evaluated on coincident points here
        if eps > 0.0:
            cases.append((2, eps, _collinear(N, 2, 3), [0, N - 1]))
            cases.append((3, eps, _collinear(N, 3, 4), [0, N - 1]))
    x = np.sort(inputs.uniform(5, 0, N) * 2.0 - 1.0)
    cases.append((4, 0.0, x, [0, N - 1]))      # outermost sheets: sign(x_i - x_j) all equal
    cases.append((4, 0.05, x, [0, N - 1]))
    # Ring: particle 0 at 0.3, the others within (0.01, pi - 0.01) ahead of it
    th = np.concatenate([[0.3], 0.3 + 0.01 + (np.pi - 0.02) * inputs.uniform(6, 0, N - 1)])
    cases.append((1, 0.01, th, [0]))
    return cases


@pytest.mark.parametrize("k", range(len(_same_sign_cases())))
def test_scale_equals_force_magnitude_when_pair_terms_share_a_sign(api, k):
    model, eps, q, rows = _same_sign_cases()[k]
    N = q.size // _dim(model)
    f = api.force(model, q, eps).reshape(_dim(model), N)[:, rows]
    a = api.force_abs(model, q, eps).reshape(_dim(model), N)[:, rows]
    _, ar = api.rows_abs(model, q, rows, eps)
    assert np.all(np.abs(f) > 0.0)
    np.testing.assert_allclose(a, np.abs(f), rtol=1e-13, atol=0.0)
    np.testing.assert_allclose(ar, np.abs(f), rtol=1e-13, atol=0.0)


@pytest.mark.parametrize("th_i,lo,hi,which", [(0.0, 0.05, np.pi - 0.05, "sin"),
                                              (np.pi / 2, -np.pi / 2 + 0.05, np.pi / 2 - 0.05, "cos")])
def test_hmf_scale_equals_force_magnitude_where_one_mean_field_term_vanishes(api, th_i, lo, hi, which):
    """HMF force f_i = cos(th_i) My - sin(th_i) Mx (Eq. 6).  At th_i = 0 only the My
    term is left, and with every sin(th_j) > 0 the scale, the sum of |cos th_i sin th_j|
    + |sin th_i cos th_j| over j divided by N, equals |f_i|; at th_i = pi/2 the Mx term
    with every cos(th_j) > 0 (cos(pi/2) is 6e-17, not 0, hence the tolerance)."""
    N = 41
    th = np.concatenate([[th_i], lo + (hi - lo) * inputs.uniform(8, 0, N - 1)])
    f = api.force(0, th, 0.0)[0]
    a = api.force_abs(0, th, 0.0)[0]
    _, ar = api.rows_abs(0, th, [0], 0.0)
    np.testing.assert_allclose([a, ar[0, 0]], abs(f), rtol=1e-13, atol=0.0)
    # the other term's sum must not leak in: it is of the same size here
    other = np.abs(np.cos(th) if which == "sin" else np.sin(th)).sum() / N
    assert other > 0.1 * abs(f)


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.01), (2, 1e-3), (3, 1e-3), (4, 0.0), (4, 0.05)])
def test_force_magnitude_is_bounded_by_the_scale(api, model, eps):
    """Triangle inequality on a random state, both copies of the scale."""
    N = 200
    q, _ = inputs.default_state(model, N, 77)
    f = np.abs(api.force(model, q, eps)).reshape(_dim(model), N)
    a = api.force_abs(model, q, eps).reshape(_dim(model), N)
    rows = np.arange(0, N, 7)
    _, ar = api.rows_abs(model, q, rows, eps)
    assert np.all(f <= a * (1 + 1e-14))
    assert np.all(f[:, rows] <= ar * (1 + 1e-14))
    # and not vacuous: the scale is within a modest factor of the force on average
    assert np.median(a) < 1e3 * np.median(f) + 1e-300


# Planted mistakes: (substring of md_oracle.c, replacement).  Each sits in one copy of
# the scale (ora_force_abs or ora_force_rows) for one model and component.
MUTATIONS = [
    ("      out[i] = c * s;", "      out[i] = 2.0 * c * s;"),                               # Ring, force_abs
    ("      if (out_abs) out_abs[r] = c * sa;", "      if (out_abs) out_abs[r] = 2.0 * c * sa;"),  # Ring, rows
    ("        sy += fabs(dy) / s;\n      }\n      out[i] = 2.0 * sx / (double)N;",              # 2D x
     "        sy += fabs(dy) / s;\n      }\n      out[i] = 4.0 * sx / (double)N;"),
    ("        sy += fabs(dy) / s;\n      }\n      out[i] = 2.0 * sx / (double)N;\n      out[N + i] = 2.0 * sy / (double)N;",
     "        sy += fabs(dy) / s;\n      }\n      out[i] = 2.0 * sx / (double)N;\n      out[N + i] = 2.0 * sx / (double)N;"),
    ("        out_abs[r] = 2.0 * ax / (double)N;", "        out_abs[r] = ax / (double)N;"),    # 2D x, rows
    ("        out_abs[nrows + r] = 2.0 * ay / (double)N;", "        out_abs[nrows + r] = 3.0 * ay / (double)N;"),
    ("      out[2 * N + i] = sz / (double)N;", "      out[2 * N + i] = 2.0 * sz / (double)N;"),  # 3D z
    ("        out_abs[2 * nrows + r] = az / (double)N;", "        out_abs[2 * nrows + r] = ay / (double)N;"),
    ("      out[i] = s / (double)N;", "      out[i] = s / (double)(N - 1);"),                   # sheets
    ("      if (out_abs) out_abs[r] = a / (double)N;", "      if (out_abs) out_abs[r] = 2.0 * a / (double)N;"),
    ("      out[i] = (fabs(cos(q[i])) * as + fabs(sin(q[i])) * ac) / (double)N;",            # HMF: swapped sums
     "      out[i] = (fabs(cos(q[i])) * ac + fabs(sin(q[i])) * as) / (double)N;"),
    ("      if (out_abs) out_abs[r] = (fabs(cos(t)) * as + fabs(sin(t)) * ac) / (double)N;",
     "      if (out_abs) out_abs[r] = (fabs(cos(t)) * as + fabs(sin(t)) * ac) / (double)(2 * N);"),
]


def _pins_hold(api):
    try:
        for k in range(len(_same_sign_cases())):
            test_scale_equals_force_magnitude_when_pair_terms_share_a_sign(api, k)
        for args in [(0.0, 0.05, np.pi - 0.05, "sin"), (np.pi / 2, -np.pi / 2 + 0.05, np.pi / 2 - 0.05, "cos")]:
            test_hmf_scale_equals_force_magnitude_where_one_mean_field_term_vanishes(api, *args)
        for model, eps in [(0, 0.0), (1, 0.01), (2, 1e-3), (3, 1e-3), (4, 0.0), (4, 0.05)]:
            test_force_magnitude_is_bounded_by_the_scale(api, model, eps)
    except AssertionError:
        return False
    return True


def test_planted_scale_mistakes_are_caught(api, tmp_path):
    src = open(SRC).read()
    assert _pins_hold(api)  # the unmodified oracle passes
    for k, (old, new) in enumerate(MUTATIONS):
        assert src.count(old) == 1, old
        path = tmp_path / f"mut{k}.c"
        path.write_text(src.replace(old, new))
        so = tmp_path / f"libmut{k}.so"
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               str(path), "-o", str(so), "-lm"])
        assert not _pins_hold(Api(ctypes.CDLL(str(so)))), f"mutation {k} not caught: {new.strip()}"

"""Contexts driven concurrently from several host threads (the binding releases the
GIL in every library call), each on its own stream: results are bitwise those of the
same contexts run one after the other, errors stay per thread and per context, and
the allocator registry and one-time kernel set-up see no races."""
import threading

import numpy as np
import pytest

from paper_1212_0262_gb300 import MDError, System, inputs

pytestmark = pytest.mark.gpu

CASES = [(0, 20011, 0.0, 0.1), (1, 3001, 0.01, 0.05), (2, 2049, 1e-3, 0.01), (3, 1500, 1e-2, 0.01),
         (4, 2500, 0.0, 0.01), (1, 1024, 0.01, 0.05)]


def _run(case, prec, out, k):
    model, N, eps, dt = case
    with System(model, N, eps, dt, 5 + k, precision=prec) as s:
        q, p = inputs.default_state(model, N, 100 + k)
        s.set_state(q, p)
        for n in (7, 4, 17, 9):  # graphs captured and replayed in both ping-pong parities
            s.step(n)
        out[k] = (s.get_state(), s.energy())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_threads_match_sequential_runs(prec):
    seq = [None] * len(CASES)
    for k, c in enumerate(CASES):
        _run(c, prec, seq, k)
    for rep in range(4):  # contexts created, captured into graphs and freed while others run
        par = [None] * len(CASES)
        errors = []

        def worker(k):
            try:
                _run(CASES[k], prec, par, k)
            except Exception as e:  # reported below
                errors.append((k, repr(e)))

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(CASES))]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert not errors, (rep, errors)
        for k in range(len(CASES)):
            (qa, pa), ea = seq[k]
            (qb, pb), eb = par[k]
            assert np.array_equal(qa, qb) and np.array_equal(pa, pb), (rep, k)
            assert ea == eb, (rep, k)


def test_errors_stay_with_their_thread_and_context():
    """A failing call in one thread leaves the other thread's context and its last
    error untouched."""
    good = System(1, 512, 0.01, 0.05, 1)
    msgs = {}

    def bad():
        s = System(4, 100, 0.0, 0.01, 1)
        try:
            s.grad(2)
        except MDError as e:
            msgs["bad"] = str(e)

    def ok():
        good.step(5)
        msgs["good"] = good.energy()

    ts = [threading.Thread(target=bad), threading.Thread(target=ok)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=120)
    assert "eps > 0" in msgs["bad"]
    assert np.isfinite(sum(msgs["good"]))
    good.close()

"""Failures injected on the host (no GPU fault): an allocator hook that fails or hands
out misaligned blocks, allocation failures in the middle of a run, and a non-finite
state.  The library reports MD_ENOMEM / MD_ENONFINITE with a message, frees what it
made, and the context or the process stays usable."""
import ctypes

import numpy as np
import pytest

from paper_1212_0262_gb300 import MDError, System, binding as B, inputs
from paper_1212_0262_gb300.allocator import use_cuda_allocator

pytestmark = pytest.mark.gpu

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Hook:
    """An allocator hook over PyTorch's caching allocator that fails on request or
    hands out blocks shifted off the 256-byte alignment."""

    def __init__(self, fail_after=None, misalign=False):
        self.fail_after, self.misalign = fail_after, misalign
        self.count, self.live = 0, {}
        self.cbs = (_ALLOC_T(self._alloc), _FREE_T(self._free))

    def _alloc(self, nbytes, _user):
        import torch

        self.count += 1
        if self.fail_after is not None and self.count > self.fail_after:
            return None
        base = int(torch.cuda.caching_allocator_alloc(int(nbytes) + 256, torch.cuda.current_device()))
        user = base + (16 if self.misalign else 0)
        self.live[user] = base
        return user

    def _free(self, ptr, _user):
        import torch

        base = self.live.pop(ptr, None)
        if base is not None:
            torch.cuda.caching_allocator_delete(base)

    def install(self):
        B.check(B.load().md_set_allocator(ctypes.cast(self.cbs[0], ctypes.c_void_p),
                                          ctypes.cast(self.cbs[1], ctypes.c_void_p), None))


@pytest.fixture(autouse=True)
def _restore_allocator():
    yield
    use_cuda_allocator()


@pytest.mark.parametrize("hook", [Hook(fail_after=0), Hook(misalign=True), Hook(fail_after=2)])
def test_init_fails_cleanly_when_allocation_fails(hook):
    hook.install()
    with pytest.raises(MDError) as e:
        System(2, 4096, 1e-3, 0.01, 1)
    assert e.value.code == B.MD_ENOMEM and "alloc" in str(e.value)
    assert not hook.live  # every block the library got was handed back
    use_cuda_allocator()
    with System(2, 4096, 1e-3, 0.01, 1) as s:
        s.step(2)


def test_allocation_failure_mid_run_is_reported_and_recoverable():
    """md_init succeeds; the first stage's buffers (mirrors, partials) cannot be had:
    md_step reports MD_ENOMEM; with allocation working again the same context steps
    and matches a fresh one."""
    hook = Hook(fail_after=6)
    hook.install()
    s = System(1, 3000, 0.01, 0.05, 4, precision="mixed")
    q, p = inputs.default_state(1, 3000, 9)
    s.set_state(q, p)
    with pytest.raises(MDError) as e:
        s.step(3)
    assert e.value.code == B.MD_ENOMEM
    hook.fail_after = None
    s.set_state(q, p)
    s.step(3)
    with System(1, 3000, 0.01, 0.05, 4, precision="mixed") as ref:
        ref.set_state(q, p)
        ref.step(3)
        assert np.array_equal(s.get_state()[0], ref.get_state()[0])
    s.close()
    assert not hook.live


@pytest.mark.parametrize("model", [0, 1, 2])
def test_non_finite_state_is_reported(model):
    N = 2000
    with System(model, N, {0: 0.0, 1: 0.01, 2: 1e-3}[model], 0.01, 1) as s:
        q, p = inputs.default_state(model, N, 5)
        bad = p.copy()
        bad[17] = np.nan
        s.set_state(q, bad)
        with pytest.raises(MDError) as e:
            s.energy()
        assert e.value.code == B.MD_ENONFINITE
        s.set_state(q, p)
        assert np.isfinite(sum(s.energy()))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("model", [1, 2, 3, 4])
def test_non_finite_position_is_reported(model, bad):
    """A NaN or infinite position (not only momentum) makes V non-finite, so md_energy
    answers MD_ENONFINITE; the 2D potential's renormalised product falls back to the
    plain sum of logarithms on such a row instead of returning a finite number."""
    N = 1000
    eps = {1: 0.01, 2: 1e-3, 3: 1e-3, 4: 0.0}[model]
    with System(model, N, eps, 0.01, 1) as s:
        q, p = inputs.default_state(model, N, 5)
        for i in (0, 517, N - 1):  # first row, a middle row, the last row of the last tile
            qb = q.copy()
            qb[i] = bad
            s.set_state(qb, p)
            with pytest.raises(MDError) as e:
                s.energy()
            assert e.value.code == B.MD_ENONFINITE, (i, str(e.value))
        s.set_state(q, p)
        assert np.isfinite(sum(s.energy()))


def test_eps_below_the_floor_is_rejected():
    """Softenings below 1e-30 (where a softened square distance could leave the normal
    FP32 range the kernels divide in) are refused by md_init and md_set_eps."""
    for model in (1, 2, 3):
        with pytest.raises(MDError) as e:
            System(model, 64, 1e-31, 0.01, 1)
        assert e.value.code == B.MD_EINVAL
    with System(2, 64, 1e-30, 0.01, 1) as s:
        with pytest.raises(MDError):
            s.set_eps(5e-324)
        s.set_eps(1e-3)
    with System(4, 64, 0.0, 0.01, 1) as s:
        with pytest.raises(MDError):
            s.set_eps(1e-40)
        s.set_eps(0.0)

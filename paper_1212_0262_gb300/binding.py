"""ctypes binding of libmd (include/md.h): same names, argument marshalling only.

Every computation happens in the CUDA library.  If libmd.so has not been built
(``__graft_entry__.build()`` or ``python -m paper_1212_0262_gb300.build``), the
first use raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmd.so")
PEAKS_PATH = os.path.join(_PKG, "libmdpeaks.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "md.h")

_lock = threading.Lock()
_lib = None
_peaks = None


def _constants() -> dict[str, int]:
    """The #define constants of md.h (parsed, so the header is the single source)."""
    consts = {}
    with open(HEADER) as fh:
        for m in re.finditer(r"^#define\s+(MD_[A-Z0-9_]+)\s+(-?\d+)", fh.read(), re.M):
            consts[m.group(1)] = int(m.group(2))
    return consts


globals().update(_constants())

_c = ctypes
_P = _c.c_void_p
_D = _c.POINTER(_c.c_double)
_SIGS = {
    "md_init": (_P, [_c.c_int, _c.c_int64, _c.c_double, _c.c_double, _c.c_uint64]),
    "md_free": (None, [_P]),
    "md_last_error": (_c.c_char_p, [_P]),
    "md_last_status": (_c.c_int, []),
    "md_set_precision": (_c.c_int, [_P, _c.c_int]),
    "md_set_stream": (_c.c_int, [_P, _P]),
    "md_set_dt": (_c.c_int, [_P, _c.c_double]),
    "md_set_eps": (_c.c_int, [_P, _c.c_double]),
    "md_set_tuning": (_c.c_int, [_P, _c.c_char_p, _c.c_int64]),
    "md_force_kernel": (_c.c_int, [_P]),
    "md_set_ic": (_c.c_int, [_P, _c.c_int, _D, _c.c_uint64]),
    "md_set_state": (_c.c_int, [_P, _P, _P]),
    "md_get_state": (_c.c_int, [_P, _P, _P]),
    "md_set_state_device": (_c.c_int, [_P, _P, _P]),
    "md_get_state_device": (_c.c_int, [_P, _P, _P]),
    "md_step": (_c.c_int, [_P, _c.c_int64]),
    "md_stage": (_c.c_int, [_P, _c.c_double, _c.c_double]),
    "md_yoshida": (None, [_D]),
    "md_force": (_c.c_int, [_P, _P]),
    "md_force_device": (_c.c_int, [_P, _P]),
    "md_energy": (_c.c_int, [_P, _D, _D]),
    "md_magnetization": (_c.c_int, [_P, _D, _D]),
    "md_grad": (_c.c_int, [_P, _c.c_int, _c.c_int64, _c.c_int, _P, _P, _D, _D]),
    "md_tangent_step": (_c.c_int, [_P, _c.c_int64, _P, _P]),
    "md_lyapunov": (_c.c_int, [_P, _c.c_int64, _c.c_int64, _P, _P, _D]),
    "md_set_allocator": (_c.c_int, [_P, _P, _P]),
    "md_potential_noalloc": (_c.c_int, [_c.c_int, _c.c_int64, _c.c_double, _P, _P, _P]),
    "md_shard_range": (_c.c_int, [_c.c_int, _c.c_int64, _c.c_int, _c.c_int, _P, _P]),
    "md_shard_init": (_P, [_c.c_int, _c.c_int64, _c.c_double, _c.c_double, _c.c_uint64, _c.c_int, _c.c_int]),
    "md_shard_begin": (_c.c_int, [_P]),
    "md_shard_stage": (_c.c_int, [_P, _c.c_double, _c.c_double]),
    "md_shard_buffer": (_c.c_int, [_P, _P, _P, _P]),
    "md_shard_exchange": (_c.c_int, [_P, _c.c_int]),
    "md_shard_step": (_c.c_int, [_P, _c.c_int, _c.c_int64]),
    "md_shard_force": (_c.c_int, [_P, _P]),
    "md_synchronize": (_c.c_int, [_P]),
    "md_launch_count": (_c.c_int64, [_P]),
    "md_batch_init": (_P, [_c.c_int, _P, _P, _P, _P, _P]),
    "md_batch_free": (None, [_P]),
    "md_batch_set_precision": (_c.c_int, [_P, _c.c_int]),
    "md_batch_set_stream": (_c.c_int, [_P, _P]),
    "md_batch_step": (_c.c_int, [_P, _c.c_int64]),
    "md_batch_set_tuning": (_c.c_int, [_P, _c.c_int, _c.c_double, _c.c_int]),
    "md_batch_get_tuning": (_c.c_int, [_P, _P, _P, _P]),
    "md_batch_autotune": (_c.c_int, [_P, _D]),
    "md_batch_force": (_c.c_int, [_P, _P]),
    "md_batch_energy": (_c.c_int, [_P, _P, _P]),
    "md_batch_get_state": (_c.c_int, [_P, _c.c_int, _P, _P]),
    "md_batch_set_state": (_c.c_int, [_P, _c.c_int, _P, _P]),
    "md_batch_last_error": (_c.c_char_p, [_P]),
    "md_batch_launch_count": (_c.c_int64, [_P]),
}


class MDError(RuntimeError):
    """A libmd call returned a nonzero status."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"libmd error {code}: {msg}")
        self.code = code


def load():
    """Load libmd.so (raises if it is missing: no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(nvcc, sm_103a); the CUDA library is the only implementation")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def load_peaks():
    global _peaks
    with _lock:
        if _peaks is None:
            if not os.path.exists(PEAKS_PATH):
                raise RuntimeError(f"{PEAKS_PATH} is missing: build it with __graft_entry__.build()")
            lib = ctypes.CDLL(PEAKS_PATH)
            lib.mdp_pipe_rates.restype = ctypes.c_int
            lib.mdp_pipe_rates.argtypes = [_D, ctypes.c_int]
            _peaks = lib
    return _peaks


def __getattr__(name):
    # md_* functions resolve lazily, so importing this module never needs a GPU
    if name.startswith("md_"):
        return getattr(load(), name)
    raise AttributeError(name)


def check(rc: int, handle=None, batch: bool = False) -> None:
    """Raise MDError for a nonzero status, with the library's message."""
    if rc != 0:
        lib = load()
        msg = (lib.md_batch_last_error(handle) if batch else lib.md_last_error(handle)) or b""
        raise MDError(rc, msg.decode(errors="replace"))

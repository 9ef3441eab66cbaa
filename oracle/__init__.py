"""FP64 CPU oracle for the long-range MD method of arXiv 1212.0262.

TEST INFRASTRUCTURE ONLY.  This package may be imported, called or linked only
by ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``.  The product library never loads it,
and it shares no code with the CUDA path.

The arithmetic lives in ``md_oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module only compiles it on demand and marshals numpy arrays through ctypes.
Each wrapper names the section or equation of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HMF, RING, GRAV2D, GRAV3D, SHEET1D, HARMONIC = 0, 1, 2, 3, 4, 9
OBS_KINETIC, OBS_MAGNETIZATION = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile md_oracle.c into liboracle.so with gcc (-O2 -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.POINTER(ctypes.c_double)
            sig = {
                "ora_yoshida": (None, [P]),
                "ora_magnetization": (None, [i64, P, P, P]),
                "ora_force_hmf": (None, [i64, P, P]),
                "ora_force_hmf_pairwise": (None, [i64, P, P]),
                "ora_potential_hmf": (d, [i64, P]),
                "ora_potential_hmf_pairwise": (d, [i64, P]),
                "ora_force": (None, [i32, i64, d, P, P]),
                "ora_potential": (d, [i32, i64, d, P]),
                "ora_kinetic": (d, [i64, P]),
                "ora_force_abs": (None, [i32, i64, d, P, P]),
                "ora_force_rows": (None, [i32, i64, d, P, ctypes.POINTER(ctypes.c_int64), i64, P, P]),
                "ora_force_sheet_f32": (None, [i64, P, P]),
                "ora_step": (i32, [i32, i64, d, d, i64, P, P]),
                "ora_hvp": (None, [i32, i64, d, P, P, P]),
                "ora_hvp_hmf_meanfield": (None, [i64, P, P, P]),
                "ora_dforce_deps": (None, [i32, i64, d, P, P]),
                "ora_grad": (i32, [i32, i64, d, d, i64, i32, P, P, P, P, P, P]),
                "ora_observable_after": (d, [i32, i64, d, d, i64, i32, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def dim(model: int) -> int:
    return 2 if model == GRAV2D else 3 if model == GRAV3D else 1


def yoshida() -> np.ndarray:
    """(B0, B1, D0, D1) of Eq. 4, from the closed form of the triple jump."""
    c = np.zeros(4)
    _load().ora_yoshida(_p(c))
    return c


def magnetization(q) -> tuple[float, float]:
    """(Mx, My) of Eq. 7."""
    q = _arr(q)
    mx, my = ctypes.c_double(), ctypes.c_double()
    _load().ora_magnetization(q.size, _p(q), ctypes.byref(mx), ctypes.byref(my))
    return mx.value, my.value


def force(model: int, q, eps: float = 0.0) -> np.ndarray:
    """Forces at q: Eq. 6 (HMF), minus the gradient of Eq. 1 (Ring), Eq. 3 (2D) or of
    the softened 3D gravitational potential (GRAV3D)."""
    q = _arr(q)
    f = np.empty_like(q)
    _load().ora_force(model, q.size // dim(model), eps, _p(q), _p(f))
    return f


def force_sheet_f32(q) -> np.ndarray:
    """1D-sheet force at eps = 0 with every sign decided on the FP32-rounded
    positions (the FP32 pair kernel's precision for that decision)."""
    q = _arr(q)
    f = np.empty_like(q)
    _load().ora_force_sheet_f32(q.size, _p(q), _p(f))
    return f


def force_hmf_pairwise(q) -> np.ndarray:
    """HMF force from the pair sum of Eq. 2 (O(N^2))."""
    q = _arr(q)
    f = np.empty_like(q)
    _load().ora_force_hmf_pairwise(q.size, _p(q), _p(f))
    return f


def potential(model: int, q, eps: float = 0.0) -> float:
    """V of Eq. 5 (HMF), Eq. 1 (Ring), Eq. 3 (2D) or the 3D gravitational potential,
    with i<j pair sums."""
    q = _arr(q)
    return _load().ora_potential(model, q.size // dim(model), eps, _p(q))


def potential_hmf_pairwise(q) -> float:
    """HMF V from the pair sum of Eq. 2."""
    q = _arr(q)
    return _load().ora_potential_hmf_pairwise(q.size, _p(q))


def kinetic(p) -> float:
    """K = (1/2) sum p^2."""
    p = _arr(p)
    return _load().ora_kinetic(p.size, _p(p))


def energy(model: int, q, p, eps: float = 0.0) -> float:
    return kinetic(p) + potential(model, q, eps)


def force_abs(model: int, q, eps: float = 0.0) -> np.ndarray:
    """sum_j |f_ij| per particle and component (scale of the force sum)."""
    q = _arr(q)
    out = np.empty_like(q)
    _load().ora_force_abs(model, q.size // dim(model), eps, _p(q), _p(out))
    return out


def force_rows(model: int, q, rows, eps: float = 0.0, with_abs: bool = False):
    """Forces on the listed particles only, shape (dim, len(rows)); with_abs also
    returns sum_j |f_ij| for those rows."""
    q = _arr(q)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(dim(model) * rows.size)
    ab = np.empty_like(out)
    _load().ora_force_rows(model, q.size // dim(model), eps, _p(q),
                           rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size, _p(out), _p(ab))
    if with_abs:
        return out.reshape(dim(model), rows.size), ab.reshape(dim(model), rows.size)
    return out.reshape(dim(model), rows.size)


def step(model: int, q, p, eps: float, dt: float, nsteps: int) -> tuple[np.ndarray, np.ndarray]:
    """nsteps of the Sec. 3 step list (Eq. 4 splitting); returns new (q, p)."""
    q = _arr(q).copy()
    p = _arr(p).copy()
    rc = _load().ora_step(model, q.size // dim(model), eps, dt, nsteps, _p(q), _p(p))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    return q, p


def hvp(model: int, q, v, eps: float = 0.0) -> np.ndarray:
    """J(q) v with J = df/dq, from the pair terms."""
    q, v = _arr(q), _arr(v)
    out = np.empty_like(q)
    _load().ora_hvp(model, q.size // dim(model), eps, _p(q), _p(v), _p(out))
    return out


def hvp_hmf_meanfield(q, v) -> np.ndarray:
    """HMF J(q) v in mean-field form (Eqs. 6-7)."""
    q, v = _arr(q), _arr(v)
    out = np.empty_like(q)
    _load().ora_hvp_hmf_meanfield(q.size, _p(q), _p(v), _p(out))
    return out


def dforce_deps(model: int, q, eps: float) -> np.ndarray:
    """df/d(eps) at q."""
    q = _arr(q)
    out = np.empty_like(q)
    _load().ora_dforce_deps(model, q.size // dim(model), eps, _p(q), _p(out))
    return out


def grad(model: int, q0, p0, eps: float, dt: float, nsteps: int, obs: int = OBS_KINETIC):
    """Discrete-adjoint gradient of the final observable: (value, gq, gp, geps)."""
    q0, p0 = _arr(q0), _arr(p0)
    gq, gp = np.empty_like(q0), np.empty_like(p0)
    ge, val = ctypes.c_double(), ctypes.c_double()
    rc = _load().ora_grad(model, q0.size // dim(model), eps, dt, nsteps, obs, _p(q0), _p(p0),
                          _p(gq), _p(gp), ctypes.byref(ge), ctypes.byref(val))
    if rc != 0:
        raise ValueError(f"oracle grad failed ({rc})")
    return val.value, gq, gp, ge.value


def observable_after(model: int, q0, p0, eps: float, dt: float, nsteps: int,
                     obs: int = OBS_KINETIC) -> float:
    """Observable of the state reached after nsteps from (q0, p0)."""
    q0, p0 = _arr(q0), _arr(p0)
    return _load().ora_observable_after(model, q0.size // dim(model), eps, dt, nsteps, obs,
                                        _p(q0), _p(p0))

"""Python objects over the C ABI: one simulated system, one ensemble.

Only argument marshalling lives here; each method is one libmd call.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as B

MODELS = {"hmf": 0, "ring": 1, "grav2d": 2, "2d": 2, "grav3d": 3, "3d": 3, "sheet1d": 4, "sheets": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}


def _model(m) -> int:
    return MODELS[m.lower()] if isinstance(m, str) else int(m)


def _prec(p) -> int:
    return PRECISIONS[p.lower()] if isinstance(p, str) else int(p)


def yoshida() -> np.ndarray:
    """(B0, B1, D0, D1) of Eq. 4 as used by md_step."""
    c = np.zeros(4)
    B.load().md_yoshida(c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return c


def stage_schedule(nsteps: int):
    """The (b, d) stage coefficients that md_step(nsteps) runs, in order."""
    B0, B1, D0, D1 = yoshida()
    out = []
    for s in range(nsteps):
        out += [((B0 if s == 0 else 2 * B0), D0), (B1, D1), (B1, D0)]
    if nsteps:
        out.append((B0, 0.0))
    return out


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class System:
    """N particles of one model (md_init .. md_free)."""

    def __init__(self, model, N: int, eps: float = 0.0, dt: float = 0.1, seed: int = 0,
                 precision="fp64"):
        lib = B.load()
        self.model = _model(model)
        self.N = int(N)
        self.dim = {2: 2, 3: 3}.get(self.model, 1)
        self._dt = float(dt)
        h = lib.md_init(self.model, self.N, float(eps), float(dt), int(seed) & (2**64 - 1))
        if not h:
            raise B.MDError(lib.md_last_status() or B.MD_EINVAL, (lib.md_last_error(None) or b"").decode())
        self._h = ctypes.c_void_p(h)
        self.set_precision(precision)

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None):
            B.load().md_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc: int) -> None:
        B.check(rc, self._h)

    # -- configuration
    def set_precision(self, precision) -> None:
        self._chk(B.load().md_set_precision(self._h, _prec(precision)))

    def set_dt(self, dt: float) -> None:
        self._chk(B.load().md_set_dt(self._h, float(dt)))
        self._dt = float(dt)

    def set_tuning(self, key: str, value: int) -> None:
        self._chk(B.load().md_set_tuning(self._h, key.encode(), int(value)))

    @property
    def force_kernel(self) -> int:
        """MD_KERNEL_* code of the force kernel the next stage runs."""
        return int(B.load().md_force_kernel(self._h))

    def set_stream(self, stream) -> None:
        """A cudaStream_t as int, or a torch.cuda.Stream."""
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(B.load().md_set_stream(self._h, ctypes.c_void_p(int(handle or 0))))

    def set_ic(self, kind: int, params=None, seed: int = 0) -> None:
        arr = None if params is None else _f64(params)
        p = None if arr is None else arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._chk(B.load().md_set_ic(self._h, int(kind), p, int(seed) & (2**64 - 1)))

    # -- state
    def set_state(self, q, p) -> None:
        q, p = _f64(q), _f64(p)
        n = self.dim * self.N
        if q.size != n or p.size != n:
            raise ValueError(f"state arrays must have {n} elements")
        self._chk(B.load().md_set_state(self._h, _ptr(q), _ptr(p)))

    def get_state(self):
        n = self.dim * self.N
        q, p = np.empty(n), np.empty(n)
        self._chk(B.load().md_get_state(self._h, _ptr(q), _ptr(p)))
        return q, p

    def set_state_device(self, q_ptr: int, p_ptr: int) -> None:
        """Device-to-device copy queued on the context's stream: whatever writes q and p
        must be ordered before it (the same stream through set_stream, or a synchronize)."""
        self._chk(B.load().md_set_state_device(self._h, ctypes.c_void_p(q_ptr), ctypes.c_void_p(p_ptr)))

    def get_state_device(self, q_ptr: int, p_ptr: int) -> None:
        self._chk(B.load().md_get_state_device(self._h, ctypes.c_void_p(q_ptr), ctypes.c_void_p(p_ptr)))

    # -- dynamics and observables
    def step(self, nsteps: int = 1) -> None:
        self._chk(B.load().md_step(self._h, int(nsteps)))

    def stage(self, b: float, d: float) -> None:
        """One fused force + kick(b dt) + drift(d dt) stage (d == 0: kick only)."""
        self._chk(B.load().md_stage(self._h, float(b), float(d)))

    def synchronize(self) -> None:
        self._chk(B.load().md_synchronize(self._h))

    def force(self) -> np.ndarray:
        f = np.empty(self.dim * self.N)
        self._chk(B.load().md_force(self._h, _ptr(f)))
        return f

    def force_device(self, f_ptr: int) -> None:
        self._chk(B.load().md_force_device(self._h, ctypes.c_void_p(f_ptr)))

    def energy(self):
        k, v = ctypes.c_double(), ctypes.c_double()
        self._chk(B.load().md_energy(self._h, ctypes.byref(k), ctypes.byref(v)))
        return k.value, v.value

    def magnetization(self):
        mx, my = ctypes.c_double(), ctypes.c_double()
        self._chk(B.load().md_magnetization(self._h, ctypes.byref(mx), ctypes.byref(my)))
        return mx.value, my.value

    def grad(self, nsteps: int, observable: int = 0, checkpoint_every: int = 20):
        """(value, grad_q, grad_p, grad_eps) of the observable after nsteps."""
        n = self.dim * self.N
        gq, gp = np.empty(n), np.empty(n)
        ge, val = ctypes.c_double(), ctypes.c_double()
        self._chk(B.load().md_grad(self._h, int(observable), int(nsteps), int(checkpoint_every),
                                   _ptr(gq), _ptr(gp), ctypes.byref(ge), ctypes.byref(val)))
        return val.value, gq, gp, ge.value

    def set_eps(self, eps: float) -> None:
        self._chk(B.load().md_set_eps(self._h, float(eps)))

    def tangent_step(self, nsteps: int, dq, dp):
        """Advance the state nsteps steps with a tangent vector; returns the new (dq, dp)."""
        dq, dp = _f64(dq).copy(), _f64(dp).copy()
        self._chk(B.load().md_tangent_step(self._h, int(nsteps), _ptr(dq), _ptr(dp)))
        return dq, dp

    def lyapunov(self, nsteps: int, renorm_every: int = 10, seed: int = 0, dt: float | None = None) -> float:
        """Largest Lyapunov exponent estimate (md_lyapunov): a seeded random tangent
        vector carried along nsteps steps (advancing the state), renormalised on the
        device every renorm_every steps; the mean log growth rate per unit time."""
        from . import inputs

        n = self.dim * self.N
        d = inputs.uniform(seed, 0, 2 * n) - 0.5
        dq, dp = np.ascontiguousarray(d[:n]), np.ascontiguousarray(d[n:])
        total = ctypes.c_double()
        self._chk(B.load().md_lyapunov(self._h, int(nsteps), int(renorm_every), _ptr(dq), _ptr(dp),
                                       ctypes.byref(total)))
        step_dt = dt if dt is not None else self._dt
        return total.value / (nsteps * step_dt)

    @property
    def launch_count(self) -> int:
        return int(B.load().md_launch_count(self._h))


class Ensemble:
    """Independent Ring / 2D systems advanced together (md_batch_*)."""

    def __init__(self, models, Ns, eps, dts, seeds, precision="mixed"):
        lib = B.load()
        self.nsys = len(Ns)
        self.models = np.ascontiguousarray([_model(m) for m in models], dtype=np.int32)
        self.Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        self._eps = _f64(eps)
        self._dts = _f64(dts)
        self._seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        h = lib.md_batch_init(self.nsys, _ptr(self.models), _ptr(self.Ns), _ptr(self._eps), _ptr(self._dts),
                              _ptr(self._seeds))
        if not h:
            raise B.MDError(lib.md_last_status() or B.MD_EINVAL, (lib.md_last_error(None) or b"").decode())
        self._h = ctypes.c_void_p(h)
        self.set_precision(precision)

    def close(self) -> None:
        if getattr(self, "_h", None):
            B.load().md_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc: int) -> None:
        B.check(rc, self._h, batch=True)

    def set_precision(self, precision) -> None:
        self._chk(B.load().md_batch_set_precision(self._h, _prec(precision)))

    def set_stream(self, stream) -> None:
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(B.load().md_batch_set_stream(self._h, ctypes.c_void_p(int(handle or 0))))

    def step(self, nsteps: int = 1) -> None:
        self._chk(B.load().md_batch_step(self._h, int(nsteps)))

    def set_tuning(self, r: int, split: float, ctas_per_sm: int = 0) -> None:
        """r = 0: Newton's-third-law kernels (mixed default); r = 4 or 8: one-sided."""
        self._chk(B.load().md_batch_set_tuning(self._h, int(r), float(split), int(ctas_per_sm)))

    @property
    def tuning(self):
        """(r, split, ctas_per_sm) of the batched launches."""
        r, cps = ctypes.c_int(), ctypes.c_int()
        split = ctypes.c_double()
        self._chk(B.load().md_batch_get_tuning(self._h, ctypes.byref(r), ctypes.byref(split), ctypes.byref(cps)))
        return r.value, split.value, cps.value

    def autotune(self) -> float:
        """Pick the fastest kernel shape; returns its force-launch time in ms."""
        ms = ctypes.c_double()
        self._chk(B.load().md_batch_autotune(self._h, ctypes.byref(ms)))
        return ms.value

    def force(self, systems=None):
        """Forces of the listed systems (default: all) at their current positions, from
        one force-only launch of the ensemble kernels; a dict system -> array."""
        systems = range(self.nsys) if systems is None else [int(s) for s in systems]
        out = {s: np.empty((2 if self.models[s] == 2 else 1) * int(self.Ns[s])) for s in systems}
        ptrs = (ctypes.c_void_p * self.nsys)()
        for s, a in out.items():
            ptrs[s] = a.ctypes.data
        self._chk(B.load().md_batch_force(self._h, ptrs))
        return out

    def energy(self):
        k, v = np.empty(self.nsys), np.empty(self.nsys)
        self._chk(B.load().md_batch_energy(self._h, _ptr(k), _ptr(v)))
        return k, v

    def get_state(self, s: int):
        n = (2 if self.models[s] == 2 else 1) * int(self.Ns[s])
        q, p = np.empty(n), np.empty(n)
        self._chk(B.load().md_batch_get_state(self._h, int(s), _ptr(q), _ptr(p)))
        return q, p

    def set_state(self, s: int, q, p) -> None:
        q, p = _f64(q), _f64(p)
        self._chk(B.load().md_batch_set_state(self._h, int(s), _ptr(q), _ptr(p)))

    @property
    def launch_count(self) -> int:
        return int(B.load().md_batch_launch_count(self._h))


def shard_range(model, N: int, rank: int, nranks: int):
    """Rows [lo, hi) of rank `rank` of `nranks` (md_shard_range)."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    B.check(B.load().md_shard_range(_model(model), int(N), int(rank), int(nranks), ctypes.byref(lo),
                                    ctypes.byref(hi)))
    return lo.value, hi.value


class ShardGroup:
    """One system split by rows among `nranks` shard contexts held by this process
    (md_shard_*): the paper's multi-GPU schemes (Sec. 3.1 last paragraph, Sec. 3.2
    Fig. 2) with the exchange done by md_shard_exchange.  `devices` (optional) puts
    rank r's context on device devices[r]; by default all ranks share the current
    device."""

    def __init__(self, model, N: int, eps: float, dt: float, seed: int, nranks: int, precision="fp64",
                 devices=None):
        import torch

        lib = B.load()
        self.model, self.N, self.nranks = _model(model), int(N), int(nranks)
        self.dim = {2: 2, 3: 3}.get(self.model, 1)
        self.ranges = [shard_range(self.model, self.N, r, self.nranks) for r in range(self.nranks)]
        self._ctx = (ctypes.c_void_p * self.nranks)()
        prev = torch.cuda.current_device() if devices else None
        try:
            for r in range(self.nranks):
                if devices:
                    torch.cuda.set_device(devices[r])
                h = lib.md_shard_init(self.model, self.N, float(eps), float(dt), int(seed) & (2**64 - 1), r,
                                      self.nranks)
                if not h:
                    self.close()
                    raise B.MDError(lib.md_last_status() or B.MD_EINVAL, (lib.md_last_error(None) or b"").decode())
                self._ctx[r] = h
        finally:
            if devices:
                torch.cuda.set_device(prev)
        self.set_precision(precision)

    def close(self) -> None:
        if getattr(self, "_ctx", None) is not None:
            for r in range(self.nranks):
                if self._ctx[r]:
                    B.load().md_free(ctypes.c_void_p(self._ctx[r]))
                    self._ctx[r] = None
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _h(self, r):
        return ctypes.c_void_p(self._ctx[r])

    def _chk(self, rc: int, r: int = 0) -> None:
        B.check(rc, self._h(r))

    def set_precision(self, precision) -> None:
        for r in range(self.nranks):
            self._chk(B.load().md_set_precision(self._h(r), _prec(precision)), r)

    def set_tuning(self, key: str, value: int) -> None:
        for r in range(self.nranks):
            self._chk(B.load().md_set_tuning(self._h(r), key.encode(), int(value)), r)

    def begin(self) -> None:
        """md_shard_begin on every rank, then the exchange."""
        lib = B.load()
        for r in range(self.nranks):
            self._chk(lib.md_shard_begin(self._h(r)), r)
        self._chk(lib.md_shard_exchange(self._ctx, self.nranks))

    def step(self, nsteps: int = 1) -> None:
        self._chk(B.load().md_shard_step(self._ctx, self.nranks, int(nsteps)))

    def stage(self, b: float, d: float) -> None:
        """One fused stage on every rank, then the exchange (md_shard_begin first when needed)."""
        lib = B.load()
        for r in range(self.nranks):
            self._chk(lib.md_shard_stage(self._h(r), float(b), float(d)), r)
        self._chk(lib.md_shard_exchange(self._ctx, self.nranks))

    def force(self) -> np.ndarray:
        """Forces on all N particles (layout of md_force), each rank's rows from its shard."""
        f = np.empty((self.dim, self.N))
        for r, (lo, hi) in enumerate(self.ranges):
            fr = np.empty(self.dim * (hi - lo))
            self._chk(B.load().md_shard_force(self._h(r), _ptr(fr)), r)
            f[:, lo:hi] = fr.reshape(self.dim, hi - lo)
        return f.reshape(-1)

    def get_state(self):
        q, p = np.empty((self.dim, self.N)), np.empty((self.dim, self.N))
        for r, (lo, hi) in enumerate(self.ranges):
            n = self.dim * (hi - lo)
            qr, pr = np.empty(n), np.empty(n)
            self._chk(B.load().md_get_state(self._h(r), _ptr(qr), _ptr(pr)), r)
            q[:, lo:hi], p[:, lo:hi] = qr.reshape(self.dim, -1), pr.reshape(self.dim, -1)
        return q.reshape(-1), p.reshape(-1)

    def set_state(self, q, p) -> None:
        """Every rank's rows of the whole-system arrays q, p (then begin and exchange)."""
        q, p = _f64(q).reshape(self.dim, self.N), _f64(p).reshape(self.dim, self.N)
        for r, (lo, hi) in enumerate(self.ranges):
            qr, pr = np.ascontiguousarray(q[:, lo:hi]), np.ascontiguousarray(p[:, lo:hi])
            self._chk(B.load().md_set_state(self._h(r), _ptr(qr), _ptr(pr)), r)
        self.begin()

    def buffer(self, r: int):
        """(device pointer, segment offset, segment bytes) of rank r's exchange buffer."""
        buf, off, nb = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_size_t()
        self._chk(B.load().md_shard_buffer(self._h(r), ctypes.byref(buf), ctypes.byref(off), ctypes.byref(nb)), r)
        return buf.value, off.value, nb.value

    def synchronize(self) -> None:
        for r in range(self.nranks):
            self._chk(B.load().md_synchronize(self._h(r)), r)

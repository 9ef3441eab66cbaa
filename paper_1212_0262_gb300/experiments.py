"""The accuracy experiments of Sec. 4 on synthetic input: relative energy error
dE(t) = |(E(t) - E0) / E0| of runs started at rest from homogeneous states
(HMF and Ring: theta uniform on [-pi, pi)) or from a uniform annulus
(2D: R1 = 1.0, R2 = 1.5), through the library's C ABI.

The paper plots these curves (its Figs. 3, 5, 7, 8) for a double-precision CPU
code and for its GPU codes; its claims are that the GPU error is of the same
order as the double-precision one and that FP32 pair forces do not spoil it.
"""
from __future__ import annotations

import numpy as np

from . import inputs
from .system import System

# the paper's parameters (Sec. 4 and the captions of Figs. 3, 5, 7)
SETUPS = {
    "hmf": dict(model=0, eps=0.0, dt=0.1),
    "ring": dict(model=1, eps=1e-3, dt=0.005),
    "grav2d": dict(model=2, eps=1e-3, dt=0.005),
}


def initial_state(model: int, N: int, seed: int):
    """Homogeneous at rest (HMF, Ring) or uniform annulus at rest (2D)."""
    if model == 2:
        return inputs.annulus_state(N, seed, 1.0, 1.5)
    return inputs.uniform_rest(N, seed)


def energy_error_series(name: str, N: int, nsteps: int, every: int, precision: str = "fp64", seed: int = 1):
    """Times and dE(t) sampled every `every` steps, plus (K, V) at each sample."""
    cfg = SETUPS[name]
    q, p = initial_state(cfg["model"], N, seed)
    with System(cfg["model"], N, cfg["eps"], cfg["dt"], seed, precision=precision) as s:
        s.set_state(q, p)
        k0, v0 = s.energy()
        e0 = k0 + v0
        t, de, kv = [0.0], [0.0], [(k0, v0)]
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            s.step(n)
            done += n
            k, v = s.energy()
            t.append(done * cfg["dt"])
            de.append(abs((k + v - e0) / e0))
            kv.append((k, v))
    return np.array(t), np.array(de), np.array(kv)

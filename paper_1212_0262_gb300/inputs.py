"""Seeded synthetic initial conditions (host side, numpy).

This module holds no arithmetic of the method: it only draws the initial states
that both the CUDA path and the CPU oracle start from.  The device-side
generator behind ``md_init`` implements the same recipe independently, and a
test compares the two.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based: the k-th draw for a seed
is the SplitMix64 output mix(seed + (k + 1) * 0x9E3779B97F4A7C15), i.e. the
k-th output of the sequential generator started at state ``seed``.
A uniform is (x >> 11) * 2^-53 in [0, 1).  A Gaussian uses two consecutive
uniforms u1, u2 (Box-Muller 1958): sqrt(-2 log(1 - u1)) cos(2 pi u2).

Draw order: all positions first (counters 0 .. dim*N - 1; the disk uses two
counters per particle, the ball three), then all momenta.  Affine maps are evaluated as
(hi - lo) * u + lo with two separate roundings.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_PI = 2.0 * np.pi

# initial-condition kinds (match the MD_IC_* codes of the C ABI)
IC_WATERBAG = 0   # HMF: theta ~ U[th_lo, th_hi), p ~ U[p_lo, p_hi)
IC_RING = 1       # Ring: theta ~ U[-pi, pi), p ~ N(0, sigma^2)
IC_DISK = 2       # 2D: uniform unit disk, p ~ N(0, sigma^2) per component
IC_ANNULUS = 3    # 2D: uniform annulus R1 <= r < R2, at rest
IC_UNIFORM_REST = 4  # angle models: theta ~ U[-pi, pi), at rest
IC_BALL = 5       # 3D: uniform unit ball, p ~ N(0, sigma^2) per component


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given 0-based counters (uint64 array)."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from counters start .. start + n - 1."""
    x = splitmix64(seed, np.arange(start, start + n, dtype=np.uint64))
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, start: int, n: int) -> np.ndarray:
    """n standard normals; normal k uses counters start + 2k and start + 2k + 1."""
    u = uniform(seed, start, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(_TWO_PI * u2)


def _affine(u: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return (hi - lo) * u + lo


def waterbag(N: int, seed: int, th_lo=-1.0, th_hi=1.0, p_lo=-1.2, p_hi=1.2):
    """HMF water-bag: theta ~ U[th_lo, th_hi), p ~ U[p_lo, p_hi)."""
    q = _affine(uniform(seed, 0, N), th_lo, th_hi)
    p = _affine(uniform(seed, N, N), p_lo, p_hi)
    return q, p


def ring_state(N: int, seed: int, sigma=0.5):
    """Ring: theta ~ U[-pi, pi), p ~ N(0, sigma^2)."""
    q = _affine(uniform(seed, 0, N), -np.pi, np.pi)
    p = sigma * gaussian(seed, N, N)
    return q, p


def disk_state(N: int, seed: int, sigma=0.3):
    """2D: uniform in the unit disk (r = sqrt(u1), phi = 2 pi u2), p ~ N(0, sigma^2)."""
    u = uniform(seed, 0, 2 * N)
    r = np.sqrt(u[0::2])
    phi = _TWO_PI * u[1::2]
    q = np.concatenate([r * np.cos(phi), r * np.sin(phi)])
    p = sigma * gaussian(seed, 2 * N, 2 * N)
    return q, p


def annulus_state(N: int, seed: int, r1=1.0, r2=1.5):
    """2D at rest, uniform in the annulus r1 <= r < r2 (area-uniform)."""
    u = uniform(seed, 0, 2 * N)
    r = np.sqrt((r2 * r2 - r1 * r1) * u[0::2] + r1 * r1)
    phi = _TWO_PI * u[1::2]
    q = np.concatenate([r * np.cos(phi), r * np.sin(phi)])
    return q, np.zeros(2 * N)


def ball_state(N: int, seed: int, sigma=0.3):
    """3D: uniform in the unit ball (r = u1^(1/3), cos(polar angle) = 1 - 2 u2,
    azimuth = 2 pi u3, counters 3i .. 3i + 2), p ~ N(0, sigma^2) per component
    (x block, then y, then z)."""
    u = uniform(seed, 0, 3 * N)
    r = np.cbrt(u[0::3])
    ct = 1.0 - 2.0 * u[1::3]
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    phi = _TWO_PI * u[2::3]
    q = np.concatenate([r * st * np.cos(phi), r * st * np.sin(phi), r * ct])
    p = sigma * gaussian(seed, 3 * N, 3 * N)
    return q, p


def sheet_state(N: int, seed: int, x_lo=-1.0, x_hi=1.0, p_lo=-0.5, p_hi=0.5):
    """1D sheets, water-bag: x ~ U[x_lo, x_hi), p ~ U[p_lo, p_hi) (the HMF recipe's
    counters and maps with the sheet model's intervals)."""
    return waterbag(N, seed, x_lo, x_hi, p_lo, p_hi)


def uniform_rest(N: int, seed: int):
    """Angle models at rest: theta ~ U[-pi, pi), p = 0."""
    return _affine(uniform(seed, 0, N), -np.pi, np.pi), np.zeros(N)


def default_state(model: int, N: int, seed: int):
    """Per-model default initial state: water-bag (HMF), ring_state, disk_state, ball_state,
    sheet_state."""
    if model == 0:
        return waterbag(N, seed)
    if model == 1:
        return ring_state(N, seed)
    if model == 2:
        return disk_state(N, seed)
    if model == 3:
        return ball_state(N, seed)
    if model == 4:
        return sheet_state(N, seed)
    raise ValueError(f"unknown model {model}")


def ensemble_sizes(nsys: int, seed: int, n_lo=4096, n_hi=65536) -> np.ndarray:
    """Log-uniform system sizes: N_s = floor(n_lo * (n_hi/n_lo)^u_s), u_s = uniform(seed, s)."""
    u = uniform(seed, 0, nsys)
    return np.floor(n_lo * (n_hi / n_lo) ** u).astype(np.int64)

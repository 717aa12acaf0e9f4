"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds random-number generation only, none of the transform's
arithmetic.  The generator is SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used in its
counter form: draw i of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``,
so any slice of a stream can be produced independently.

Doubles in [0, 1) take the top 53 bits: ``(u >> 11) * 2**-53``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = float(2.0 ** -53)

BASE_SEED = 150107350


def config_seed(k: int) -> int:
    """Seed of workload k (one seed per benchmark configuration)."""
    return BASE_SEED + int(k)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _chunks(count: int, chunk: int = 1 << 24):
    for s in range(0, count, chunk):
        yield s, min(chunk, count - s)


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    for s, c in _chunks(count):
        out[s:s + c] = (splitmix64(seed, start + s, c) >> np.uint64(11)).astype(np.float64) * _TWO_M53
    return out


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    """i.i.d. uniform[-1, 1): 2 * U[0,1) - 1 (exact in FP64)."""
    return uniform01(seed, count, start) * 2.0 - 1.0


def normal(seed: int, count: int) -> np.ndarray:
    """i.i.d. standard normal by Box-Muller on pairs of uniform draws."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def complex_field(shape, seed: int, dist: str = "uniform") -> np.ndarray:
    """complex128 array of ``shape``; element i takes draws 2i (re), 2i+1 (im)."""
    n = int(np.prod(shape))
    if dist == "uniform":
        v = uniform_pm1(seed, 2 * n)
    elif dist == "normal":
        v = normal(seed, 2 * n)
    else:
        raise ValueError("dist must be 'uniform' or 'normal'")
    return v.view(np.complex128).reshape(shape)


def plane_wave(Na: int, Nb: int, Nc: int, k0) -> np.ndarray:
    """exp(+2 pi i (a ka0/Na + b kb0/Nb + c kc0/Nc)) on [Na][Nb][Nc].

    The phase index is reduced exactly in integers before the cosine/sine, so
    the input is accurate to one rounding per component."""
    ka0, kb0, kc0 = k0
    a = np.arange(Na, dtype=np.int64)[:, None, None]
    b = np.arange(Nb, dtype=np.int64)[None, :, None]
    c = np.arange(Nc, dtype=np.int64)[None, None, :]
    N = Na * Nb * Nc
    t = ((a * ka0) % Na) * (N // Na) + ((b * kb0) % Nb) * (N // Nb) + ((c * kc0) % Nc) * (N // Nc)
    t = t % N
    ang = 2.0 * np.pi * (t.astype(np.float64) / float(N))
    return (np.cos(ang) + 1j * np.sin(ang)).astype(np.complex128)


def batch_shapes(seed: int, count: int = 64):
    """Sizes of the batched workload: drawn uniformly from four 3-D shapes."""
    menu = [(48, 48, 48), (64, 64, 64), (96, 96, 96), (100, 108, 120)]
    u = splitmix64(seed, 0, count)
    return [menu[int(x % np.uint64(4))] for x in u]

"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays them out; it holds none of the
transform arithmetic.  Every workload of the paper is "a random band-limited
signal" (Sec. 4.4): harmonic coefficients drawn at random and, where a map is
needed, synthesised from them by an inverse transform that the caller supplies.

Conventions
-----------
* Harmonic coefficients are stored as ``flm[l, m + L - 1]`` (complex128), i.e. a
  ``[L, 2L-1]`` array; entries with ``|m| > l`` or ``l < |spin|`` are zero.
* "Complex Gaussian of variance v" means the real and imaginary parts are each
  N(0, v/2).
* The reality condition (real spin-0 signals) is ``f[l, -m] = (-1)^m conj f[l, m]``
  with ``f[l, 0]`` real and N(0, v).
* Wigner coefficients are stored as ``flmn[n + N - 1, l, m + L - 1]``.
* Every generator takes a ``numpy.random.Generator``; ``rng_for`` builds the
  canonical one from ``(seed, config, item)``.
"""
from __future__ import annotations

import numpy as np

SEED = 20240202


def rng_for(config: int, item: int = 0, seed: int = SEED) -> np.random.Generator:
    """The generator used for workload ``config`` and map/field ``item``."""
    return np.random.default_rng([seed, config, item])


def power_law(l: np.ndarray) -> np.ndarray:
    """Variance (l+1)^-2 used by the sphere workloads."""
    return (l + 1.0) ** -2


def white(l: np.ndarray) -> np.ndarray:
    return np.ones_like(l, dtype=np.float64)


def flm_random(L: int, rng: np.random.Generator, spin: int = 0, reality: bool = False,
               variance=power_law) -> np.ndarray:
    """Random band-limited harmonic coefficients ``[L, 2L-1]``."""
    out = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    for l in range(abs(spin), L):
        v = float(variance(np.asarray(float(l))))
        if reality:
            out[l, L - 1] = rng.normal(0.0, np.sqrt(v))
            if l > 0:
                re = rng.normal(0.0, np.sqrt(v / 2), size=l)
                im = rng.normal(0.0, np.sqrt(v / 2), size=l)
                pos = re + 1j * im
                m = np.arange(1, l + 1)
                out[l, L - 1 + m] = pos
                out[l, L - 1 - m] = ((-1.0) ** m) * np.conj(pos)
        else:
            re = rng.normal(0.0, np.sqrt(v / 2), size=2 * l + 1)
            im = rng.normal(0.0, np.sqrt(v / 2), size=2 * l + 1)
            out[l, L - 1 - l:L + l] = re + 1j * im
    return out


def flmn_random(L: int, N: int, rng: np.random.Generator, variance=white) -> np.ndarray:
    """Random complex Wigner coefficients ``[2N-1, L, 2L-1]`` (zero where |m|>l or |n|>l)."""
    out = np.zeros((2 * N - 1, L, 2 * L - 1), dtype=np.complex128)
    for n in range(-(N - 1), N):
        for l in range(abs(n), L):
            v = float(variance(np.asarray(float(l))))
            re = rng.normal(0.0, np.sqrt(v / 2), size=2 * l + 1)
            im = rng.normal(0.0, np.sqrt(v / 2), size=2 * l + 1)
            out[n + N - 1, l, L - 1 - l:L + l] = re + 1j * im
    return out


def pixels_random(shape, rng: np.random.Generator, complex_: bool = False) -> np.ndarray:
    """Unstructured (not band-limited) samples, used to pin linear operators exactly."""
    x = rng.normal(size=shape)
    if complex_:
        x = x + 1j * rng.normal(size=shape)
    return x


def flmp_random(L: int, P: int, rng: np.random.Generator, reality: bool = True) -> np.ndarray:
    """Ball coefficients ``[P, L, 2L-1]`` with variance (l+1)^-2 (p+1)^-2."""
    out = np.zeros((P, L, 2 * L - 1), dtype=np.complex128)
    for p in range(P):
        out[p] = flm_random(L, rng, reality=reality,
                            variance=lambda l, p=p: (l + 1.0) ** -2 * (p + 1.0) ** -2)
    return out

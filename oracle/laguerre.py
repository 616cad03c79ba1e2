"""Fourier-Laguerre radial transform and the spherical-Laguerre transform (oracle; test only).

Definitions (Sec. 2.3):
* K_p(r) = sqrt(p!/(p+2)!) exp(-r/(2 tau)) tau^(-3/2) L^(2)_p(r/tau)           (Eq. 6)
* forward f_p = int_0^inf r^2 f(r) K_p(r) dr                                   (Eq. 7)
* inverse f(r) = sum_{p<P} f_p K_p(r)                                          (Eq. 8)
* Z_lmp = K_p Y_lm, forward Z (Eq. 10) and inverse (Eq. 11) on the ball.

The radial integral is evaluated exactly for band-limited signals (p < P) by P-point
generalised Gauss-Laguerre quadrature with weight x^2 e^-x: nodes x_i are the roots of
L^(2)_P, r_i = tau x_i, weights w_i, and omega_i = tau^3 w_i e^{x_i} so that
f_p = sum_i omega_i K_p(r_i) f(r_i).  (The radial band-limit is read as p = 0..P-1.)
Nodes, weights and K_p(r_i) are computed in 40-digit arithmetic (mpmath) from the
three-term Laguerre recurrence and Newton-polished roots, then rounded to float64.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import mpmath as mp
from scipy.special import roots_genlaguerre

ALPHA = 2


def _lag_all(P: int, x):
    """[L^(2)_0(x), ..., L^(2)_P(x)] by the three-term recurrence (mpmath)."""
    out = [mp.mpf(1), 1 + ALPHA - x]
    for p in range(1, P):
        out.append(((2 * p + 1 + ALPHA - x) * out[p] - (p + ALPHA) * out[p - 1]) / (p + 1))
    return out[:P + 1]


@lru_cache(maxsize=16)
def quadrature(P: int, tau: float = 1.0):
    """(r_i, omega_i, K[i, p] = K_p(r_i)) as float64 arrays."""
    with mp.workdps(40):
        x0, _ = roots_genlaguerre(P, ALPHA)
        xs = []
        for x in x0:
            x = mp.mpf(float(x))
            for _ in range(60):
                Ls = _lag_all(P, x)
                # d/dx L^(a)_P = -L^(a+1)_{P-1};  L^(a+1)_{P-1} = sum_{k<P} L^(a)_k
                dL = -mp.fsum(Ls[:P])
                step = Ls[P] / dL
                x -= step
                if abs(step) < mp.mpf(10) ** -36 * (1 + abs(x)):
                    break
            xs.append(x)
        r = np.zeros(P)
        om = np.zeros(P)
        K = np.zeros((P, P))
        t = mp.mpf(tau)
        gam = mp.gamma(P + ALPHA + 1) / mp.factorial(P)
        for i, x in enumerate(xs):
            Ls = _lag_all(P + 1, x)
            w = gam * x / ((P + 1) ** 2 * Ls[P + 1] ** 2)
            r[i] = float(t * x)
            om[i] = float(t ** 3 * w * mp.exp(x))
            for p in range(P):
                norm = mp.sqrt(mp.factorial(p) / mp.factorial(p + 2))
                K[i, p] = float(norm * mp.exp(-x / 2) * t ** mp.mpf(-1.5) * Ls[p])
    return r, om, K


def radial_forward(f_r: np.ndarray, P: int, tau: float = 1.0) -> np.ndarray:
    """Eq. 7: f_r[i, ...] samples at r_i -> f_p[p, ...]."""
    _, om, K = quadrature(P, tau)
    return np.tensordot((om[:, None] * K).T, f_r, axes=(1, 0))


def radial_inverse(f_p: np.ndarray, P: int, tau: float = 1.0) -> np.ndarray:
    """Eq. 8: f_p[p, ...] -> samples f_r[i, ...] at the nodes r_i."""
    _, _, K = quadrature(P, tau)
    return np.tensordot(K, f_p, axes=(1, 0))


def spherical_laguerre_forward(f: np.ndarray, L: int, P: int, tau: float = 1.0,
                               spin: int = 0, samp: str = "mw") -> np.ndarray:
    """Z (Eq. 10): samples f[i, t, p] on (r_i, MW or DH grid) -> f_lmp as [P, L, 2L-1]."""
    from . import harmonic
    flm_r = np.stack([harmonic.sht_forward(f[i], L, spin, samp) for i in range(P)])
    return radial_forward(flm_r, P, tau)


def spherical_laguerre_inverse(flmp: np.ndarray, L: int, P: int, tau: float = 1.0,
                               spin: int = 0, samp: str = "mw") -> np.ndarray:
    """Z^-1 (Eq. 11): f_lmp [P, L, 2L-1] -> samples [P nodes, R rings, 2L-1] (complex)."""
    from . import harmonic
    flm_r = radial_inverse(flmp, P, tau)
    return np.stack([harmonic.sht_inverse(flm_r[i], L, spin, samp) for i in range(P)])

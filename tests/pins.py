"""Independent closed forms used to pin the oracle (test helpers; no oracle code here).

Everything here is written from textbook definitions with libraries other than the
oracle's: Wigner's explicit sum in 40-digit arithmetic, scipy's Condon-Shortley
spherical harmonics, Dirichlet-kernel interpolation and adaptive quadrature.
"""
from __future__ import annotations

import math
import warnings

import mpmath as mp
import numpy as np
from scipy import integrate
from scipy.special import sph_harm_y


def d_explicit(l: int, m: int, n: int, beta: float) -> float:
    """Wigner's explicit sum for d^l_mn(beta) (Varshalovich convention), 40 digits."""
    with mp.workdps(40):
        b = mp.mpf(beta)
        c, s = mp.cos(b / 2), mp.sin(b / 2)
        tot = mp.mpf(0)
        for k in range(0, 2 * l + 1):
            a1, a2, a3, a4 = l + n - k, k, m - n + k, l - m - k
            if min(a1, a2, a3, a4) < 0:
                continue
            tot += (-1) ** (m - n + k) * c ** (2 * l + n - m - 2 * k) * s ** (m - n + 2 * k) / (
                mp.factorial(a1) * mp.factorial(a2) * mp.factorial(a3) * mp.factorial(a4))
        pref = mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * mp.factorial(l + n) *
                       mp.factorial(l - n))
        return float(pref * tot)


def ylm_cs(l: int, m: int, theta, phi):
    """Condon-Shortley spherical harmonic from scipy (independent of the oracle)."""
    return sph_harm_y(l, m, theta, phi)


def syl_goldberg(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    """Goldberg et al. (1967) explicit spin-weighted harmonic, 40 digits."""
    with mp.workdps(40):
        th = mp.mpf(theta)
        pref = (-1) ** m * mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * (2 * l + 1) /
                                   (4 * mp.pi * mp.factorial(l + s) * mp.factorial(l - s)))
        tot = mp.mpf(0)
        for r in range(0, l - s + 1):
            k2 = r + s - m
            if k2 < 0 or k2 > l + s:
                continue
            tot += mp.binomial(l - s, r) * mp.binomial(l + s, k2) * (-1) ** (l - r - s) * \
                mp.cot(th / 2) ** (2 * r + s - m)
        val = pref * mp.sin(th / 2) ** (2 * l) * tot
        return complex(val) * complex(np.exp(1j * m * phi))


def dirichlet_interp(samples: np.ndarray, L: int):
    """The degree-(L-1) trigonometric interpolant through 2L-1 equispaced samples at
    theta_u = pi (2u+1)/(2L-1), as a callable (closed-form Dirichlet kernel)."""
    n = 2 * L - 1
    th = np.pi * (2.0 * np.arange(n) + 1.0) / n

    def g(theta):
        x = theta - th
        num = np.sin(n * x / 2.0)
        den = n * np.sin(x / 2.0)
        ker = np.where(np.abs(den) < 1e-300, 1.0, num / np.where(den == 0, 1.0, den))
        return np.sum(samples * ker)
    return g


def quad_complex(fun, a, b):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        re, _ = integrate.quad(lambda x: fun(x).real, a, b, epsabs=1e-14, epsrel=1e-13, limit=400)
        im, _ = integrate.quad(lambda x: fun(x).imag, a, b, epsabs=1e-14, epsrel=1e-13, limit=400)
    return re + 1j * im


def rot_zyz(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Active rotation R_z(alpha) R_y(beta) R_z(gamma) as a 3x3 matrix."""
    def rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])

    def ry(b):
        c, s = math.cos(b), math.sin(b)
        return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])
    return rz(alpha) @ ry(beta) @ rz(gamma)

"""Scale-discretised directional wavelet dictionary (oracle; test infrastructure only).

Follows App. A of the paper:
* s(t) = exp(-1/(1-t^2)) on (-1, 1), zero elsewhere (Eq. A3);
* s_lambda(t) = s(2 lambda/(lambda-1) (t - 1/lambda) - 1), support [1/lambda, 1] (Eq. A2);
* k_lambda(t) = int_t^1 s_lambda(u)^2/u du / int_{1/lambda}^1 s_lambda(u)^2/u du (Eq. A4),
  equal to 1 for t <= 1/lambda and 0 for t >= 1;
* kappa_lambda(t) = sqrt(k_lambda(t/lambda) - k_lambda(t)) (Eq. A5), the difference evaluated as
  the single integral of s_lambda^2/u over [t/lambda, t] (same quantity, no cancellation);
* azimuthal tiling zeta_lm = xi mu sqrt(2^-q binom(q, (q-m)/2)) (Eq. A6) with xi = 1 for
  even N-1 and i otherwise, mu = [1 - (-1)^(N+m)]/2, q = min(N-1, l - [1 + (-1)^(N+l)]/2);
* Psi^j_lm = sqrt((2l+1)/(8 pi^2)) kappa^j(l) zeta_lm (Eq. A9, radial factor dropped);
* Phi_l0 = sqrt((2l+1)/(4 pi)) eta(l / lambda^J0) with eta = sqrt(k_lambda) (App. A.1).

Readings where the paper is ambiguous (listed in the design notes):
* kappa^j(l) = kappa_lambda(l / lambda^j), j increasing with frequency, so scale j lives
  on l in (lambda^(j-1), lambda^(j+1)) as Sec. 3.3 (Eq. 38) states;
* J = the smallest integer with lambda^J >= L, scales j = J0..J;
* multiresolution band-limits L_j = min(ceil(lambda^(j+1)), L), N_j = min(N, L_j), and
  the scaling band-limit L_Phi = ceil(lambda^J0) (Phi vanishes for l >= lambda^J0).
The normalising integral of k_lambda uses adaptive Gauss-Kronrod quadrature (QUADPACK).
"""
from __future__ import annotations

import math
import warnings
from functools import lru_cache

import numpy as np
from scipy import integrate


def s_bump(t: float) -> float:
    if t <= -1.0 or t >= 1.0:
        return 0.0
    return math.exp(-1.0 / (1.0 - t * t))


def s_lambda(t: float, lam: float) -> float:
    return s_bump(2.0 * lam / (lam - 1.0) * (t - 1.0 / lam) - 1.0)


def _integrand(u: float, lam: float) -> float:
    return s_lambda(u, lam) ** 2 / u


@lru_cache(maxsize=64)
def _k_norm(lam: float) -> float:
    return _quad(1.0 / lam, lam)


def _quad(t: float, lam: float, upper: float = 1.0) -> float:
    """int_t^upper s_lambda(u)^2/u du (QUADPACK; it reports round-off once it reaches ~1e-16
    relative accuracy, which is the goal)."""
    if upper <= t:
        return 0.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _ = integrate.quad(_integrand, t, upper, args=(lam,), epsabs=0.0, epsrel=1.2e-14,
                                limit=500)
    return val


@lru_cache(maxsize=200000)
def k_lambda(t: float, lam: float) -> float:
    if t <= 1.0 / lam:
        return 1.0
    if t >= 1.0:
        return 0.0
    return _quad(t, lam) / _k_norm(lam)


@lru_cache(maxsize=200000)
def kappa_lambda(t: float, lam: float) -> float:
    """kappa_lambda(t) = sqrt(k_lambda(t/lambda) - k_lambda(t)) (Eq. A5).

    With Eq. A4 the difference is one integral, int_{t/lambda}^{t} s_lambda(u)^2/u du over the
    normalisation; it is evaluated that way so that values near the support edges keep their
    relative precision (k(t/lambda) - k(t) computed as a difference of two numbers close to 1
    underflows to 0 where the true value is ~1e-17)."""
    a = max(t / lam, 1.0 / lam)
    b = min(t, 1.0)
    if b <= a:
        return 0.0
    return math.sqrt(_quad(a, lam, b) / _k_norm(lam))


def eta_lambda(t: float, lam: float) -> float:
    return math.sqrt(k_lambda(t, lam))


def _ceil_pow(lam: float, e: int) -> int:
    v = lam ** e
    r = round(v)
    return int(r) if abs(v - r) < 1e-9 * max(1.0, v) else int(math.ceil(v))


def n_scales_max(L: int, lam: float) -> int:
    """J: the smallest integer with lambda^J >= L."""
    J = 0
    while _ceil_pow(lam, J) < L:
        J += 1
    return J


def scale_bandlimits(L: int, N: int, lam: float, J0: int):
    """[(j, L_j, N_j)] for j = J0..J (multiresolution, Sec. 3.3)."""
    J = n_scales_max(L, lam)
    out = []
    for j in range(J0, J + 1):
        Lj = min(_ceil_pow(lam, j + 1), L)
        out.append((j, Lj, min(N, Lj)))
    return out


def scaling_bandlimit(L: int, lam: float, J0: int) -> int:
    return min(_ceil_pow(lam, J0), L)


def zeta(l: int, m: int, N: int) -> complex:
    """Azimuthal tiling zeta_lm (Eq. A6)."""
    xi = 1.0 if (N - 1) % 2 == 0 else 1j
    mu = (1 - (-1) ** ((N + m) % 2)) // 2
    q = min(N - 1, l - (1 + (-1) ** ((N + l) % 2)) // 2)
    if mu == 0 or q < 0 or abs(m) > q or (q - m) % 2 != 0:
        return 0.0
    return xi * math.sqrt(math.comb(q, (q - m) // 2) / 2.0 ** q)


def wavelet_filter(L: int, N: int, lam: float, j: int, spin: int = 0) -> np.ndarray:
    """Psi^j[l, n + N - 1] for l < L, |n| < N (Eq. A9)."""
    psi = np.zeros((L, 2 * N - 1), dtype=np.complex128)
    for l in range(abs(spin), L):
        kap = kappa_lambda(l / lam ** j, lam)
        if kap == 0.0:
            continue
        for n in range(-(N - 1), N):
            psi[l, n + N - 1] = math.sqrt((2 * l + 1) / (8 * math.pi ** 2)) * kap * zeta(l, n, N)
    return psi


def scaling_filter(L: int, lam: float, J0: int, spin: int = 0) -> np.ndarray:
    """Phi_l0 for l < L (App. A.1 scaling generator eta = sqrt(k))."""
    phi = np.zeros(L)
    for l in range(abs(spin), L):
        phi[l] = math.sqrt((2 * l + 1) / (4 * math.pi)) * eta_lambda(l / lam ** J0, lam)
    return phi

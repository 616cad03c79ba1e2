"""Samplings of S^2 and SO(3) (oracle; test infrastructure only).

The paper benchmarks on McEwen-Wiaux (MW) sampling (Sec. 4.4) but defers its
definition to the MW sampling theorem; the grids below are that theorem's:
colatitudes theta_t = pi (2t+1)/(2L-1), t = 0..L-1 (the last ring is the south
pole), longitudes phi_p = 2 pi p/(2L-1), p = 0..2L-2, and on SO(3) the third Euler
angle gamma_g = 2 pi g/(2N-1), g = 0..2N-2.

The transforms are also stated to be sampling agnostic, with Driscoll-Healy (DH)
sampling among the supported grids (Sec. 1).  The DH grid used here has 2L colatitude
rings at the midpoints theta_t = pi (2t+1)/(4L), t = 0..2L-1 (no pole is sampled), the
same 2L-1 longitudes and, on SO(3), the same 2N-1 angles gamma.  Its colatitude integral
is a plain weighted sum over the rings: the weights w_t are fixed by requiring
sum_t w_t cos(k theta_t) = int_0^pi cos(k theta) sin(theta) d theta for k = 0..2L-1
(2L conditions for 2L weights), which makes the rule exact for every product of two
band-limited colatitude columns (a cosine series of degree <= 2L-2).
"""
import numpy as np


def thetas(L: int) -> np.ndarray:
    return np.pi * (2.0 * np.arange(L) + 1.0) / (2.0 * L - 1.0)


def thetas_extended(L: int) -> np.ndarray:
    """The 2L-1 equispaced colatitudes of the periodic extension to [0, 2 pi)."""
    return np.pi * (2.0 * np.arange(2 * L - 1) + 1.0) / (2.0 * L - 1.0)


def phis(L: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(2 * L - 1) / (2.0 * L - 1.0)


def gammas(N: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(2 * N - 1) / (2.0 * N - 1.0)


def sin_weight(q: np.ndarray) -> np.ndarray:
    """w(q) = integral_0^pi exp(i q theta) sin(theta) d theta for integer q.

    Closed form: 2/(1-q^2) for even q, +-i pi/2 for q = +-1, 0 for other odd q.
    """
    q = np.asarray(q)
    out = np.zeros(q.shape, dtype=np.complex128)
    even = (q % 2) == 0
    out[even] = 2.0 / (1.0 - q[even].astype(np.float64) ** 2)
    out[q == 1] = 0.5j * np.pi
    out[q == -1] = -0.5j * np.pi
    return out


SAMPLINGS = ("mw", "dh")


def thetas_dh(L: int) -> np.ndarray:
    """The 2L Driscoll-Healy colatitudes pi (2t+1)/(4L)."""
    return np.pi * (2.0 * np.arange(2 * L) + 1.0) / (4.0 * L)


def rings(L: int, sampling: str = "mw") -> int:
    """Number of colatitude rings of the grid at band-limit L."""
    if sampling not in SAMPLINGS:
        raise ValueError(sampling)
    return L if sampling == "mw" else 2 * L


def thetas_for(L: int, sampling: str = "mw") -> np.ndarray:
    if sampling not in SAMPLINGS:
        raise ValueError(sampling)
    return thetas(L) if sampling == "mw" else thetas_dh(L)


def cos_sin_moment(k: np.ndarray) -> np.ndarray:
    """int_0^pi cos(k theta) sin(theta) d theta = (1 + (-1)^k)/(1 - k^2) (0 for k = 1)."""
    k = np.asarray(k)
    out = np.zeros(k.shape, dtype=np.float64)
    even = (k % 2) == 0
    out[even] = 2.0 / (1.0 - k[even].astype(np.float64) ** 2)
    return out


def dh_weights(L: int) -> np.ndarray:
    """DH colatitude weights w_t (t < 2L) from the moment conditions, by a dense solve."""
    th = thetas_dh(L)
    k = np.arange(2 * L)
    A = np.cos(np.outer(k, th))          # [k, t]
    return np.linalg.solve(A, cos_sin_moment(k))

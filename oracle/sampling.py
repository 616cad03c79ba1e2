"""McEwen-Wiaux sampling of S^2 and SO(3) (oracle; test infrastructure only).

The paper benchmarks on McEwen-Wiaux (MW) sampling (Sec. 4.4) but defers its
definition to the MW sampling theorem; the grids below are that theorem's:
colatitudes theta_t = pi (2t+1)/(2L-1), t = 0..L-1 (the last ring is the south
pole), longitudes phi_p = 2 pi p/(2L-1), p = 0..2L-2, and on SO(3) the third Euler
angle gamma_g = 2 pi g/(2N-1), g = 0..2N-2.
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

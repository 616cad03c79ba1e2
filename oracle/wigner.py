"""Wigner-d functions as trigonometric polynomials in beta (oracle; test infrastructure only).

The paper factorises D^l_mn(alpha, beta, gamma) = d^l_mn(beta) exp(-i(m alpha + n gamma))
(Sec. 5.2, Eq. 47) and leaves d^l_mn to its references; we use the standard
(Varshalovich) convention  d^l_mn(beta) = <l m| exp(-i beta J_y) |l n>,  for which
d^1_10 = -sin(beta)/sqrt 2 and d^1_11 = (1 + cos beta)/2.

Route taken here (independent of the GPU path's three-term recursion in l):
rotating J_x by a quarter turn about z gives J_y, so
    exp(-i beta J_y) = exp(-i pi/2 J_z) exp(-i beta J_x) exp(i pi/2 J_z).
J_x is a real symmetric tridiagonal matrix with the integer spectrum -l..l; with
J_x = V diag(lambda) V^T,
    d^l_mn(beta) = (-i)^(m-n) sum_j V[m, j] V[n, j] exp(-i lambda_j beta),
a trigonometric polynomial of degree l.  Its Fourier coefficients
    d^l_mn(beta) = sum_{k=-l..l} c^l_mn(k) exp(i k beta)
are what the MW algorithm needs for the exact colatitude integrals.  (The columns
of V are, up to sign, the rows of Delta^l = d^l(pi/2) used by McEwen and Wiaux.)
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from scipy.linalg import eigh_tridiagonal


@lru_cache(maxsize=1100)
def jx_eigen(l: int):
    """Integer eigenvalues (ascending, -l..l) and orthonormal eigenvectors of J_x.

    Rows of V are indexed by m + l.  J_+ |m> = sqrt((l-m)(l+m+1)) |m+1>, J_x = (J_+ + J_-)/2.
    """
    m = np.arange(-l, l + 1, dtype=np.float64)
    off = 0.5 * np.sqrt((l - m[:-1]) * (l + m[:-1] + 1.0))
    if l == 0:
        return np.zeros(1, dtype=np.int64), np.ones((1, 1))
    lam, V = eigh_tridiagonal(np.zeros(2 * l + 1), off)
    k = np.rint(lam).astype(np.int64)
    assert np.array_equal(k, np.arange(-l, l + 1)), "J_x spectrum must be -l..l"
    return k, V


def _phase(m: np.ndarray, n: np.ndarray) -> np.ndarray:
    """(-i)^(m-n) elementwise, exactly."""
    table = np.array([1.0, -1j, -1.0, 1j])
    return table[np.mod(m[:, None] - n[None, :], 4)]


def fourier_coeffs(l: int, ns=None) -> np.ndarray:
    """c^l_mn(k) as an array C[m + l, i_n, k + l] for the requested n values (default all).

    d^l_mn(beta) = sum_k C[m+l, i_n, k+l] exp(i k beta).  Entries for |n| > l are zero.
    """
    if ns is None:
        ns = np.arange(-l, l + 1)
    ns = np.asarray(ns, dtype=np.int64)
    _, V = jx_eigen(l)
    ms = np.arange(-l, l + 1)
    C = np.zeros((2 * l + 1, len(ns), 2 * l + 1), dtype=np.complex128)
    ok = np.abs(ns) <= l
    if not ok.any():
        return C
    nsv = ns[ok]
    # eigenvalue lambda_j = j - l contributes to k = -lambda_j, i.e. column j = l - k.
    Vr = V[:, ::-1]                       # Vr[:, k + l] = V[:, l - k]
    prod = Vr[:, None, :] * Vr[nsv + l][None, :, :]
    C[:, ok, :] = _phase(ms, nsv)[:, :, None] * prod
    return C


def d_matrix(l: int, beta: float) -> np.ndarray:
    """d^l_mn(beta) for all m, n as a real [2l+1, 2l+1] array (rows m+l, columns n+l)."""
    C = fourier_coeffs(l)
    k = np.arange(-l, l + 1)
    val = C @ np.exp(1j * k * beta)
    return val.real


def d_values(l: int, m: int, n: int, betas: np.ndarray) -> np.ndarray:
    """d^l_mn at several angles."""
    C = fourier_coeffs(l, [n])[m + l, 0]
    k = np.arange(-l, l + 1)
    return (np.exp(1j * np.outer(betas, k)) @ C).real

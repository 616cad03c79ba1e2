"""Spin spherical-harmonic and Wigner transforms on MW and DH sampling (oracle; test infrastructure only).

Definitions followed
--------------------
* Forward spin SHT (Sec. 2.1, Eq. 2):  f_lm = int f(omega) sY*_lm(omega) dOmega, and the
  inverse (Eq. 3): f = sum_lm f_lm sY_lm, band-limited at L.
* Forward Wigner transform (Sec. 2.2, Eq. 4): F^l_mn = int f(rho) D^l_mn(rho) dOmega(rho)
  (no conjugate), inverse (Eq. 5): f = sum (2l+1)/(8 pi^2) F^l_mn D^l*_mn.
* D^l_mn(alpha, beta, gamma) = d^l_mn(beta) exp(-i(m alpha + n gamma)) (Sec. 5.2, Eq. 47).
* ``wigner_inverse_ring``: Eq. 5 at a single colatitude, for sampled checks of large transforms.
* sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) exp(i m phi) (the MW
  convention; the paper is silent).  For s = 0 this is the Condon-Shortley Y_lm.

Algorithm (McEwen-Wiaux, which the paper's benchmark sampling refers to; Sec. 4.4):
the alpha/phi and gamma integrals are exact DFT sums over the equispaced samples
(Eq. 48's "Fourier transform" factor); the colatitude integral of a band-limited
column G(theta) against d^l_mn(theta) sin(theta) is done exactly by
  (1) extending G to [0, 2 pi) with G(2 pi - theta) = (-1)^(m+n) G(theta) (the parity
      of d^l_mn, since d^l_mn(-beta) = (-1)^(m-n) d^l_mn(beta)),
  (2) taking its 2L-1 Fourier coefficients Ghat(p) from the 2L-1 extended samples,
  (3) forming I(k) = int_0^pi G(theta) e^{i k theta} sin(theta) = sum_p Ghat(p) w(p + k)
      with the closed-form weights w of ``sampling.sin_weight``,
  (4) contracting with the Fourier coefficients of d^l_mn (``wigner.fourier_coeffs``).
All DFTs are direct O(n^2) sums written as matrix products.

Driscoll-Healy sampling (``samp="dh"``; the grid and weights of ``sampling``): the
inverse transforms evaluate the same Fourier series at the 2L DH rings, and the forward
transforms replace steps (1)-(3) by
  I(k) = sum_t w_t G(theta_t) exp(i k theta_t),
so that step (4), which is shared, yields sum_t w_t G(theta_t) d^l_mn(theta_t): the DH
quadrature of the colatitude integral, exact whenever G d^l_mn is a cosine series of
degree <= 2L-1 (every band-limited column).
"""
from __future__ import annotations

import numpy as np

from . import sampling, wigner


def _mrange(L):
    return np.arange(-(L - 1), L)


def _colatitude_integrals(G: np.ndarray, L: int, parity: np.ndarray) -> np.ndarray:
    """I[k, col] = int_0^pi G_col(theta) exp(i k theta) sin(theta) d theta for |k| <= L-1.

    G is [L, ncol] (samples on the L MW colatitudes); parity[col] = +-1 is the
    reflection sign of the column's periodic extension.
    """
    ncol = G.shape[1]
    Gext = np.zeros((2 * L - 1, ncol), dtype=np.complex128)
    Gext[:L] = G
    # theta_{2L-2-t} = 2 pi - theta_t for t = 0..L-2
    Gext[L:] = parity[None, :] * G[L - 2::-1] if L > 1 else Gext[L:]
    th = sampling.thetas_extended(L)
    p = _mrange(L)
    Fwd = np.exp(-1j * np.outer(p, th)) / (2 * L - 1)   # [p, u]
    Ghat = Fwd @ Gext                                     # [p, col]
    k = _mrange(L)
    Wk = sampling.sin_weight(k[:, None] + p[None, :])     # [k, p]
    return Wk @ Ghat


def _dh_integrals(G: np.ndarray, L: int) -> np.ndarray:
    """I[k, col] = sum_t w_t G_col(theta_t) exp(i k theta_t), |k| <= L-1, on the 2L DH rings."""
    th = sampling.thetas_dh(L)
    w = sampling.dh_weights(L)
    k = _mrange(L)
    return np.exp(1j * np.outer(k, th)) @ (w[:, None] * G)


def _integrals(G, L, parity, samp):
    return _colatitude_integrals(G, L, parity) if samp == "mw" else _dh_integrals(G, L)


def sht_inverse(flm: np.ndarray, L: int, spin: int = 0, samp: str = "mw") -> np.ndarray:
    """Inverse spin SHT (Eq. 3).  flm [L, 2L-1] -> f [R theta, 2L-1 phi] (complex), R rings."""
    ms = _mrange(L)
    Cmk = np.zeros((2 * L - 1, 2 * L - 1), dtype=np.complex128)   # [m, k]
    for l in range(abs(spin), L):
        Cl = wigner.fourier_coeffs(l, [-spin])[:, 0, :]            # [m, k] for |m|,|k| <= l
        norm = (-1.0) ** spin * np.sqrt((2 * l + 1) / (4 * np.pi))
        sl = slice(L - 1 - l, L + l)
        Cmk[sl, sl] += norm * flm[l, sl][:, None] * Cl
    th = sampling.thetas_for(L, samp)
    G = Cmk @ np.exp(1j * np.outer(ms, th))                        # [m, t]
    E = np.exp(1j * np.outer(ms, sampling.phis(L)))                 # [m, p]
    return G.T @ E


def sht_forward(f: np.ndarray, L: int, spin: int = 0, samp: str = "mw") -> np.ndarray:
    """Forward spin SHT (Eq. 2) of samples f [R, 2L-1] -> flm [L, 2L-1]."""
    ms = _mrange(L)
    E = np.exp(-1j * np.outer(sampling.phis(L), ms))                # [p, m]
    G = (2 * np.pi / (2 * L - 1)) * (np.asarray(f, dtype=np.complex128) @ E)   # [t, m]
    parity = (-1.0) ** ((ms + spin) % 2)
    I = _integrals(G, L, parity, samp)                              # [k, m]
    flm = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    for l in range(abs(spin), L):
        Cl = wigner.fourier_coeffs(l, [-spin])[:, 0, :]             # [m, k]
        sl = slice(L - 1 - l, L + l)
        norm = (-1.0) ** spin * np.sqrt((2 * l + 1) / (4 * np.pi))
        flm[l, sl] = norm * np.einsum('mk,km->m', Cl, I[sl, sl])
    return flm


def wigner_inverse(flmn: np.ndarray, L: int, N: int, samp: str = "mw") -> np.ndarray:
    """Inverse Wigner transform (Eq. 5).  flmn [2N-1, L, 2L-1] -> f [2N-1 gamma, R beta, 2L-1 alpha]."""
    ms = _mrange(L)
    ns = np.arange(-(N - 1), N)
    Cnmk = np.zeros((2 * N - 1, 2 * L - 1, 2 * L - 1), dtype=np.complex128)   # [n, m, k]
    for l in range(L):
        Cl = wigner.fourier_coeffs(l, ns)                            # [m, n, k]
        sl = slice(L - 1 - l, L + l)
        coef = (2 * l + 1) / (8 * np.pi ** 2) * flmn[:, l, sl]       # [n, m]
        Cnmk[:, sl, sl] += np.transpose(Cl, (1, 0, 2)) * coef[:, :, None]
    betas = sampling.thetas_for(L, samp)
    G = Cnmk @ np.exp(1j * np.outer(ms, betas))                      # [n, m, b]
    Ea = np.exp(1j * np.outer(ms, sampling.phis(L)))                  # [m, a]
    Eg = np.exp(1j * np.outer(ns, sampling.gammas(N)))               # [n, g]
    H = np.einsum('nmb,ma->nba', G, Ea)                              # alpha sum
    return np.einsum('nba,ng->gba', H, Eg)                           # gamma sum


def wigner_inverse_ring(flmn: np.ndarray, L: int, N: int, beta: float) -> np.ndarray:
    """The inverse Wigner transform (Eq. 5) at one colatitude beta: f(alpha_a, beta, gamma_g) as
    [2N-1 gamma, 2L-1 alpha].  The same sum as ``wigner_inverse``, evaluated at one beta: d^l_mn(beta)
    = (-i)^(m-n) sum_j V[m, j] V[n, j] exp(-i lambda_j beta) from the J_x eigenvectors (the route
    of ``wigner.fourier_coeffs``, summed at this beta), then the l, m and n sums, so a single ring
    of a large transform costs O(N L^3) multiply-adds and no [n, m, k] array."""
    ms = _mrange(L)
    ns = np.arange(-(N - 1), N)
    H = np.zeros((2 * N - 1, 2 * L - 1), dtype=np.complex128)        # [n, m]
    for l in range(L):
        ok = np.abs(ns) <= l
        nsv = ns[ok]
        _, V = wigner.jx_eigen(l)
        Vr = V[:, ::-1]                                              # column k + l: eigenvalue -k
        k = np.arange(-l, l + 1)
        d = wigner._phase(np.arange(-l, l + 1), nsv) * ((Vr * np.exp(1j * k * beta)[None, :]) @ Vr[nsv + l].T)
        sl = slice(L - 1 - l, L + l)
        H[ok, sl] += (2 * l + 1) / (8 * np.pi ** 2) * flmn[ok, l, sl] * d.T
    Ea = np.exp(1j * np.outer(ms, sampling.phis(L)))                  # [m, a]
    Eg = np.exp(1j * np.outer(ns, sampling.gammas(N)))               # [n, g]
    return Eg.T @ (H @ Ea)                                           # [g, a]


def wigner_forward(f: np.ndarray, L: int, N: int, samp: str = "mw") -> np.ndarray:
    """Forward Wigner transform (Eq. 4) of SO(3) samples f [2N-1, R, 2L-1] -> flmn."""
    ms = _mrange(L)
    ns = np.arange(-(N - 1), N)
    Ea = np.exp(-1j * np.outer(sampling.phis(L), ms))                # [a, m]
    Eg = np.exp(-1j * np.outer(sampling.gammas(N), ns))              # [g, n]
    f = np.asarray(f, dtype=np.complex128)
    G = np.einsum('gba,am->gbm', f, Ea)
    G = np.einsum('gbm,gn->nbm', G, Eg)
    G *= (2 * np.pi / (2 * L - 1)) * (2 * np.pi / (2 * N - 1))      # [n, b, m]
    parity = (-1.0) ** ((ms[None, :] + ns[:, None]) % 2)              # [n, m]
    R = G.shape[1]
    Gcols = np.transpose(G, (1, 0, 2)).reshape(R, -1)
    I = _integrals(Gcols, L, parity.reshape(-1), samp)
    I = I.reshape(2 * L - 1, 2 * N - 1, 2 * L - 1)                  # [k, n, m]
    flmn = np.zeros((2 * N - 1, L, 2 * L - 1), dtype=np.complex128)
    for l in range(L):
        Cl = wigner.fourier_coeffs(l, ns)                            # [m, n, k]
        sl = slice(L - 1 - l, L + l)
        flmn[:, l, sl] = np.einsum('mnk,knm->nm', Cl, I[sl][:, :, sl])
    return flmn

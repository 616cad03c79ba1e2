"""Directional scale-discretised wavelet transform on S^2 (oracle; test infrastructure only).

Algorithm 1 of the paper, step by step:
  analysis   f_lm = Y f;  W^Phi = Y^-1 (sqrt(4 pi/(2l+1)) Phi_l0 f_lm)               (Eq. 41, Eq. 29)
             for j: W^j = D^-1 [ (8 pi^2/(2l+1)) f_lm Psi^j*_ln ]                    (Eq. 40, Eq. 27)
  synthesis  f_lm = sqrt(4 pi/(2l+1)) Phi_l0 (Y W^Phi)_lm + sum_j sum_n (D W^j)^l_mn Psi^j_ln
             f = Y^-1 f_lm                                                            (Eq. 42)
with each scale j transformed at its own band-limits (L_j, N_j) and the scaling map at
L_Phi (multiresolution, Sec. 3.3).  The scaling map is a spin-0 function (the
axisymmetric convolution restricted to gamma = 0), so it is synthesised with spin 0;
only Y f and the final Y^-1 carry the signal's spin.
"""
from __future__ import annotations

import math

import numpy as np

from . import filters, harmonic


def _embed_slice(Lsmall: int, Lbig: int):
    return slice(Lbig - Lsmall, Lbig + Lsmall - 1)


def analysis(f: np.ndarray, L: int, N: int, lam: float, J0: int, spin: int = 0,
             reality: bool = False, samp: str = "mw"):
    """Returns ([W^j as [2N_j-1, R_j, 2L_j-1] for j = J0..J], W^Phi as [R_Phi, 2L_Phi-1]).

    R is the ring count of the sampling (``samp``: "mw" or "dh") at each band-limit."""
    flm = harmonic.sht_forward(f, L, spin, samp)
    LP = filters.scaling_bandlimit(L, lam, J0)
    wphi = harmonic.sht_inverse(scaling_coefficients(flm, L, lam, J0, spin), LP, 0, samp)
    wavs = []
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        coef = scale_coefficients(flm, L, N, lam, j, Lj, Nj, spin)
        w = harmonic.wigner_inverse(coef, Lj, Nj, samp)
        wavs.append(w.real.copy() if reality else w)
    return wavs, (wphi.real.copy() if reality else wphi)


def scaling_coefficients(flm: np.ndarray, L: int, lam: float, J0: int, spin: int = 0) -> np.ndarray:
    """The harmonic coefficients of the scaling map (Eq. 29): sqrt(4 pi/(2l+1)) Phi_l0 f_lm for
    l < L_Phi, as [L_Phi, 2L_Phi-1]; W^Phi is their spin-0 inverse SHT (Eq. 41)."""
    LP = filters.scaling_bandlimit(L, lam, J0)
    phi = filters.scaling_filter(L, lam, J0, spin)
    wphi_lm = np.zeros((LP, 2 * LP - 1), dtype=np.complex128)
    sl = _embed_slice(LP, L)
    for l in range(LP):
        wphi_lm[l] = math.sqrt(4 * math.pi / (2 * l + 1)) * phi[l] * flm[l, sl]
    return wphi_lm


def scale_coefficients(flm: np.ndarray, L: int, N: int, lam: float, j: int, Lj: int, Nj: int,
                       spin: int = 0) -> np.ndarray:
    """The Wigner coefficients of wavelet scale j (Eq. 27): (8 pi^2/(2l+1)) f_lm conj(Psi^j_ln) for
    l < L_j, |n| < N_j, as [2N_j-1, L_j, 2L_j-1]; W^j is their inverse Wigner transform (Eq. 40)."""
    psi = filters.wavelet_filter(L, N, lam, j, spin)
    coef = np.zeros((2 * Nj - 1, Lj, 2 * Lj - 1), dtype=np.complex128)
    slj = _embed_slice(Lj, L)
    for l in range(Lj):
        for n in range(-(Nj - 1), Nj):
            coef[n + Nj - 1, l] = (8 * math.pi ** 2 / (2 * l + 1)) * flm[l, slj] * \
                np.conj(psi[l, n + N - 1])
    return coef


def synthesis(wavs, wphi: np.ndarray, L: int, N: int, lam: float, J0: int, spin: int = 0,
              reality: bool = False, samp: str = "mw") -> np.ndarray:
    """Inverse of ``analysis`` (Eq. 42)."""
    flm = np.zeros((L, 2 * L - 1), dtype=np.complex128)
    LP = filters.scaling_bandlimit(L, lam, J0)
    phi = filters.scaling_filter(L, lam, J0, spin)
    wphi_lm = harmonic.sht_forward(wphi, LP, 0, samp)
    sl = _embed_slice(LP, L)
    for l in range(LP):
        flm[l, sl] += math.sqrt(4 * math.pi / (2 * l + 1)) * phi[l] * wphi_lm[l]
    for (j, Lj, Nj), w in zip(filters.scale_bandlimits(L, N, lam, J0), wavs):
        psi = filters.wavelet_filter(L, N, lam, j, spin)
        coef = harmonic.wigner_forward(w, Lj, Nj, samp)
        slj = _embed_slice(Lj, L)
        for l in range(Lj):
            acc = np.zeros(2 * Lj - 1, dtype=np.complex128)
            for n in range(-(Nj - 1), Nj):
                acc += coef[n + Nj - 1, l] * psi[l, n + N - 1]
            flm[l, slj] += acc
    f = harmonic.sht_inverse(flm, L, spin, samp)
    return f.real.copy() if reality else f


def wavelet_harmonic_coeffs(flm: np.ndarray, L: int, N: int, lam: float, J0: int, spin: int = 0):
    """The Wigner coefficients of each W^j, (8 pi^2/(2l+1)) f_lm Psi^j*_ln (Eq. 27), per scale."""
    out = []
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        psi = filters.wavelet_filter(L, N, lam, j, spin)
        coef = np.zeros((2 * Nj - 1, Lj, 2 * Lj - 1), dtype=np.complex128)
        slj = _embed_slice(Lj, L)
        for l in range(Lj):
            for n in range(-(Nj - 1), Nj):
                coef[n + Nj - 1, l] = (8 * math.pi ** 2 / (2 * l + 1)) * flm[l, slj] * \
                    np.conj(psi[l, n + N - 1])
        out.append(coef)
    return out

"""Adjoints of the directional wavelet transforms (oracle; test infrastructure only).

The transforms of Algorithm 1 are linear maps, and the gradient of a loss through a linear
map is its adjoint applied to the loss's gradient (the differentiability of Sec. 4.3).  The
adjoint A^H of A is fixed by <y, A x> = <A^H y, x> for <u, v> = Re sum_i conj(u_i) v_i over
every stored sample.  This module writes that definition out by brute force: the matrix of
the analysis operator (Eqs. 40-41) or of the synthesis operator (Eq. 42) is built column by
column by applying the oracle transform (oracle.wavelet) to unit inputs, and the adjoint is
its conjugate transpose.  Complex plans are complex-linear, so unit vectors of the complex
basis suffice; real plans (spin 0, real maps) give real matrices.  The cost is one transform
per input sample: tiny band-limits only.

Vectors are flattened in the library's layout: a map as [R][2L-1]; the wavelet side as the
scales j = J0..J concatenated, each [2N_j-1][R_j][2L_j-1], followed by nothing else; the
scaling map separately as [R_Phi][2L_Phi-1].  R is the ring count of the sampling ``samp``
(L for MW, 2L for DH) at each band-limit.
"""
from __future__ import annotations

import numpy as np

from . import filters, sampling, wavelet


def _shapes(L: int, N: int, lam: float, J0: int, samp: str = "mw"):
    scales = [(2 * Nj - 1, sampling.rings(Lj, samp), 2 * Lj - 1)
              for (_, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0)]
    LP = filters.scaling_bandlimit(L, lam, J0)
    return scales, (sampling.rings(LP, samp), 2 * LP - 1)


def _flatten(wavs, wphi, real: bool):
    v = np.concatenate([np.asarray(w).ravel() for w in wavs] + [np.asarray(wphi).ravel()])
    return v.real.copy() if real else v.astype(np.complex128)


def _split(v: np.ndarray, L: int, N: int, lam: float, J0: int, samp: str = "mw"):
    scales, sphi = _shapes(L, N, lam, J0, samp)
    wavs, o = [], 0
    for s in scales:
        n = int(np.prod(s))
        wavs.append(v[o:o + n].reshape(s))
        o += n
    return wavs, v[o:o + sphi[0] * sphi[1]].reshape(sphi)


def analysis_matrix(L: int, N: int, lam: float, J0: int, spin: int = 0, reality: bool = False,
                    samp: str = "mw") -> np.ndarray:
    """Matrix of f -> (W^j for all j, W^Phi) (Algorithm 1 analysis), columns = unit maps."""
    real = reality and spin == 0
    R = sampling.rings(L, samp)
    n_in = R * (2 * L - 1)
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, dtype=np.float64 if real else np.complex128)
        e[k] = 1.0
        wavs, wphi = wavelet.analysis(e.reshape(R, 2 * L - 1), L, N, lam, J0, spin, reality=real, samp=samp)
        cols.append(_flatten(wavs, wphi, real))
    return np.stack(cols, axis=1)


def synthesis_matrix(L: int, N: int, lam: float, J0: int, spin: int = 0, reality: bool = False,
                     samp: str = "mw") -> np.ndarray:
    """Matrix of (W^j for all j, W^Phi) -> f (Eq. 42), columns = unit coefficient arrays."""
    real = reality and spin == 0
    scales, sphi = _shapes(L, N, lam, J0, samp)
    n_in = sum(int(np.prod(s)) for s in scales) + sphi[0] * sphi[1]
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, dtype=np.float64 if real else np.complex128)
        e[k] = 1.0
        wavs, wphi = _split(e, L, N, lam, J0, samp)
        f = wavelet.synthesis(wavs, wphi, L, N, lam, J0, spin, reality=real, samp=samp)
        f = np.asarray(f)
        cols.append(f.real.ravel().copy() if real else f.ravel().astype(np.complex128))
    return np.stack(cols, axis=1)


def analysis_adjoint(gwavs, gphi, L: int, N: int, lam: float, J0: int, spin: int = 0, reality: bool = False,
                     matrix: np.ndarray | None = None, samp: str = "mw") -> np.ndarray:
    """A^H (gwavs, gphi) as a [R][2L-1] map; `matrix` may pass a cached analysis_matrix."""
    real = reality and spin == 0
    A = analysis_matrix(L, N, lam, J0, spin, reality, samp) if matrix is None else matrix
    y = _flatten(gwavs, gphi, real)
    return (A.conj().T @ y).reshape(sampling.rings(L, samp), 2 * L - 1)


def synthesis_adjoint(gf, L: int, N: int, lam: float, J0: int, spin: int = 0, reality: bool = False,
                      matrix: np.ndarray | None = None, samp: str = "mw"):
    """S^H gf as (list of [2N_j-1][R_j][2L_j-1] arrays, [R_Phi][2L_Phi-1] array)."""
    real = reality and spin == 0
    S = synthesis_matrix(L, N, lam, J0, spin, reality, samp) if matrix is None else matrix
    y = np.asarray(gf).ravel()
    y = y.real.copy() if real else y.astype(np.complex128)
    return _split(S.conj().T @ y, L, N, lam, J0, samp)

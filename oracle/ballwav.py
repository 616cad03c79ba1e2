"""Directional scale-discretised wavelet transform on the ball B^3 (oracle; test only).

Sec. 3.2 with the multiresolution of Sec. 3.3, the operators of Sec. 5.1 and the dictionary
of App. A.3-A.4, for spin-0 fields band-limited at angular L and radial P:

  analysis   f_lmp = Z f                                            (Sec. 2.3, Eq. 10)
             W^Phi = Z^-1 [ sqrt(4 pi/(2l+1)) Phi_l0p f_lmp ]       (scaling coefficients)
             W^{jj'} = Q^-1 [ (8 pi^2/(2l+1)) f_lmp Psi^{jj'*}_lnp ] (Wigner-Laguerre coefficients)
  synthesis  f_lmp = sqrt(4 pi/(2l+1)) Phi_l0p (Z W^Phi)_lmp + sum_{jj'} sum_n (Q W^{jj'})^l_mnp Psi^{jj'}_lnp
             f = Z^-1 f_lmp

with Psi^{jj'}_lnp = sqrt((2l+1)/(8 pi^2)) kappa^j(l) kappa^{j'}(p) zeta_ln (App. A.4) and
Q = K D (the Wigner transform at every radial node, then the Laguerre transform, Sec. 5.2).
Scale (j, j') lives on the MW SO(3) grid at (L_j, N_j) of the sphere transform and on the
P_j'-node Gauss-Laguerre rule, P_j' = min(ceil(nu^{j'+1}), P): kappa^{j'}(p) vanishes for
p >= nu^{j'+1}, so that rule integrates every radial product exactly.

Scaling function (the printed hybrid generator does not satisfy the admissibility
condition): |Phi_l0p|^2 (4 pi/(2l+1)) = A + B - A B with A = k_lambda(l / lambda^J0) and
B = k_nu(p / nu^J0'), wavelets for j >= J0 and j' >= J0'.  Then
sum_{jj'} kappa^j(l)^2 kappa^{j'}(p)^2 = (1 - A)(1 - B) and admissibility holds exactly.

Layouts: a field is [P nodes, L, 2L-1]; W^{jj'} is [P_j' nodes, 2N_j-1, L_j, 2L_j-1]; W^Phi
is [P, L, 2L-1].  Real fields (spin 0) return real arrays.
"""
from __future__ import annotations

import math

import numpy as np

from . import filters, harmonic, laguerre, sampling


def radial_bandlimits(P: int, nu: float, J0r: int):
    """[(j', P_j')] for j' = J0'..J' with J' the smallest integer such that nu^J' >= P."""
    Jr = filters.n_scales_max(P, nu)
    return [(jr, min(filters._ceil_pow(nu, jr + 1), P)) for jr in range(J0r, Jr + 1)]


def radial_kappa(P: int, nu: float, jr: int) -> np.ndarray:
    """kappa^{j'}(p) = kappa_nu(p / nu^{j'}) for p < P (App. A.3)."""
    return np.array([filters.kappa_lambda(p / nu ** jr, nu) for p in range(P)])


def scaling_filter(L: int, P: int, lam: float, nu: float, J0: int, J0r: int) -> np.ndarray:
    """sqrt(4 pi/(2l+1)) Phi_l0p as [P, L] (the factor that multiplies f_lmp)."""
    out = np.zeros((P, L))
    for p in range(P):
        B = filters.k_lambda(p / nu ** J0r, nu)
        for l in range(L):
            A = filters.k_lambda(l / lam ** J0, lam)
            out[p, l] = math.sqrt(max(0.0, A + B - A * B))
    return out


def _embed(Lsmall: int, Lbig: int):
    return slice(Lbig - Lsmall, Lbig + Lsmall - 1)


def analysis(f: np.ndarray, L: int, N: int, P: int, lam: float, nu: float, J0: int, J0r: int,
             tau: float = 1.0, reality: bool = True, samp: str = "mw"):
    """Returns ({(j, j'): W^{jj'}}, W^Phi); angular grids of the sampling ``samp``."""
    flmp = laguerre.spherical_laguerre_forward(f, L, P, tau, samp=samp)
    phi = scaling_filter(L, P, lam, nu, J0, J0r)
    wphi = laguerre.spherical_laguerre_inverse(flmp * phi[:, :, None], L, P, tau, samp=samp)
    wavs = {}
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        psi = filters.wavelet_filter(L, N, lam, j)
        sl = _embed(Lj, L)
        for (jr, Pj) in radial_bandlimits(P, nu, J0r):
            kap = radial_kappa(P, nu, jr)
            _, _, K = laguerre.quadrature(Pj, tau)
            out = np.zeros((Pj, 2 * Nj - 1, sampling.rings(Lj, samp), 2 * Lj - 1),
                           dtype=np.float64 if reality else np.complex128)
            for i in range(Pj):
                # radial inverse of kappa^{j'}(p) f_lmp at node r_i of the P_j' rule
                g = sum(K[i, p] * kap[p] * flmp[p] for p in range(Pj))
                coef = np.zeros((2 * Nj - 1, Lj, 2 * Lj - 1), dtype=np.complex128)
                for l in range(Lj):
                    for n in range(-(Nj - 1), Nj):
                        coef[n + Nj - 1, l] = (8 * math.pi ** 2 / (2 * l + 1)) * g[l, sl] * np.conj(psi[l, n + N - 1])
                w = harmonic.wigner_inverse(coef, Lj, Nj, samp)
                out[i] = w.real if reality else w
            wavs[(j, jr)] = out
    return wavs, (wphi.real.copy() if reality else wphi)


def synthesis(wavs, wphi: np.ndarray, L: int, N: int, P: int, lam: float, nu: float, J0: int, J0r: int,
              tau: float = 1.0, reality: bool = True, samp: str = "mw") -> np.ndarray:
    """Inverse of ``analysis``."""
    phi = scaling_filter(L, P, lam, nu, J0, J0r)
    flmp = laguerre.spherical_laguerre_forward(wphi, L, P, tau, samp=samp) * phi[:, :, None]
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        psi = filters.wavelet_filter(L, N, lam, j)
        sl = _embed(Lj, L)
        for (jr, Pj) in radial_bandlimits(P, nu, J0r):
            kap = radial_kappa(P, nu, jr)
            _, om, K = laguerre.quadrature(Pj, tau)
            W = wavs[(j, jr)]
            for i in range(Pj):
                coef = harmonic.wigner_forward(W[i], Lj, Nj, samp)
                acc = np.zeros((L, 2 * L - 1), dtype=np.complex128)
                for l in range(Lj):
                    for n in range(-(Nj - 1), Nj):
                        acc[l, sl] += coef[n + Nj - 1, l] * psi[l, n + N - 1]
                for p in range(Pj):
                    flmp[p] += kap[p] * om[i] * K[i, p] * acc
    f = laguerre.spherical_laguerre_inverse(flmp, L, P, tau, samp=samp)
    return f.real.copy() if reality else f

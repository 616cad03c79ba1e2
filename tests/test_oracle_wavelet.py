"""Pins for the oracle's wavelet transform (oracle/wavelet.py)."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import synth
from oracle import filters, harmonic, sampling, wavelet
from tests.pins import rot_zyz, ylm_cs


@pytest.mark.parametrize("L,N,lam,J0,spin,real", [(32, 4, 2.0, 0, 0, True), (16, 3, 2.0, 1, 2, False),
                                                  (12, 5, 1.5, 2, 0, True), (9, 1, 2.0, 0, 0, True)])
def test_round_trip_exact(L, N, lam, J0, spin, real):
    """Exact synthesis (Eq. 31 / Eq. 42) on band-limited signals, to machine precision (Sec. 4.4)."""
    flm = synth.flm_random(L, synth.rng_for(200, L), spin=spin, reality=real)
    f = harmonic.sht_inverse(flm, L, spin)
    if real:
        f = f.real
    W, Wp = wavelet.analysis(f, L, N, lam, J0, spin, real)
    f2 = wavelet.synthesis(W, Wp, L, N, lam, J0, spin, real)
    assert np.abs(f2 - f).max() / np.abs(f).max() < 1e-13
    if real:
        Wc, _ = wavelet.analysis(f, L, N, lam, J0, spin, False)
        assert max(np.abs(w.imag).max() for w in Wc) < 1e-13 * max(np.abs(w).max() for w in Wc)


def _sphere_quadrature(L):
    x, w = leggauss(L)
    th = np.arccos(x)
    ph = 2 * math.pi * np.arange(2 * L) / (2 * L)
    T, P = np.meshgrid(th, ph, indexing='ij')
    W = np.outer(w, np.full(2 * L, 2 * math.pi / (2 * L)))
    return T, P, W


def _synth(coef, T, P):
    out = np.zeros(T.shape, complex)
    for (l, m), c in coef.items():
        out += c * ylm_cs(l, m, T, P)
    return out


def test_directional_convolution_in_pixel_space():
    """W^j(rho) = <f, R_rho Psi^j> (Eq. 26, Eq. 14) evaluated by brute force: rotate the
    wavelet's pixel-space function with a 3x3 rotation matrix and integrate on a
    Gauss-Legendre grid, using scipy's spherical harmonics."""
    L, N, lam, J0 = 6, 3, 2.0, 1
    flm = synth.flm_random(L, synth.rng_for(201, 0), reality=True)
    f = harmonic.sht_inverse(flm, L).real
    W, Wp = wavelet.analysis(f, L, N, lam, J0, 0, True)
    T, P, Wq = _sphere_quadrature(L + 1)
    fpix = _synth({(l, m): flm[l, m + L - 1] for l in range(L) for m in range(-l, l + 1)}, T, P)
    vec = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    rng = np.random.default_rng(7)
    for (j, Lj, Nj), w in zip(filters.scale_bandlimits(L, N, lam, J0), W):
        psi = filters.wavelet_filter(L, N, lam, j)
        pcoef = {(l, n): psi[l, n + N - 1] for l in range(L) for n in range(-min(l, N - 1), min(l, N - 1) + 1)}
        for _ in range(4):
            g, b, a = rng.integers(2 * Nj - 1), rng.integers(Lj), rng.integers(2 * Lj - 1)
            R = rot_zyz(sampling.phis(Lj)[a], sampling.thetas(Lj)[b], sampling.gammas(Nj)[g])
            v = vec @ R            # rows are R^T v: the pre-image of each quadrature point
            th2 = np.arccos(np.clip(v[..., 2], -1, 1))
            ph2 = np.arctan2(v[..., 1], v[..., 0])
            rot_psi = _synth(pcoef, th2, ph2)
            ref = np.sum(Wq * fpix * np.conj(rot_psi))
            assert abs(w[g, b, a] - ref) < 1e-12 * max(1.0, np.abs(w).max())
    # scaling map: W^Phi(omega) = <f, R_omega Phi> with R_omega = R(phi, theta, 0)
    LP = filters.scaling_bandlimit(L, lam, J0)
    phi = filters.scaling_filter(L, lam, J0)
    for t in range(LP):
        for p in range(2 * LP - 1):
            R = rot_zyz(sampling.phis(LP)[p], sampling.thetas(LP)[t], 0.0)
            v = vec @ R
            th2 = np.arccos(np.clip(v[..., 2], -1, 1))
            ph2 = np.arctan2(v[..., 1], v[..., 0])
            rot_phi = _synth({(l, 0): phi[l] for l in range(L)}, th2, ph2)
            ref = np.sum(Wq * fpix * np.conj(rot_phi))
            assert abs(Wp[t, p] - ref) < 1e-12


def test_wigner_coefficients_of_wavelet_maps():
    """Eq. 27: the forward Wigner transform of W^j returns (8 pi^2/(2l+1)) f_lm Psi^j*_ln."""
    L, N, lam, J0 = 16, 4, 2.0, 1
    flm = synth.flm_random(L, synth.rng_for(202, 0), reality=True)
    f = harmonic.sht_inverse(flm, L).real
    W, _ = wavelet.analysis(f, L, N, lam, J0, 0, True)
    for (j, Lj, Nj), w, c in zip(filters.scale_bandlimits(L, N, lam, J0), W,
                                 wavelet.wavelet_harmonic_coeffs(flm, L, N, lam, J0)):
        assert np.abs(harmonic.wigner_forward(w, Lj, Nj) - c).max() < 1e-13

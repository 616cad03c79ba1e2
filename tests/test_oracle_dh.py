"""Pins for the oracle's Driscoll-Healy sampling (oracle/sampling.py, harmonic.py with samp="dh").

Each DH function is checked against something other than itself:
* the colatitude weights against Fejer's first quadrature rule in closed form (the DH
  midpoint rings are its Chebyshev nodes x_t = cos theta_t), and against the exact
  polynomial moments int_{-1}^{1} x^k dx (exact up to k = 2L-1 and no further);
* the inverse transforms against scipy's Condon-Shortley harmonics, Goldberg's spin
  harmonics and Wigner's explicit d-sum evaluated at the DH rings;
* the forward transforms on arbitrary (not band-limited) samples against the definition of
  the DH quadrature written out with the explicit harmonics (a single pixel maps to
  w_t (2 pi/(2L-1)) conj(sY_lm(theta_t, phi_p)));
* the forward transforms on band-limited data against the MW route (Fourier-space
  convolution weights, an independent algorithm) on the same function sampled on both grids.
"""
import math

import numpy as np
import pytest

import synth
from oracle import harmonic, sampling, wavelet
from tests.pins import d_explicit, syl_goldberg, ylm_cs


def fejer1(M: int) -> np.ndarray:
    """Fejer's first rule on M Chebyshev nodes cos(pi (2t+1)/(2M)) (Waldvogel 2006, Eq. 2.4)."""
    th = np.pi * (2.0 * np.arange(M) + 1.0) / (2.0 * M)
    k = np.arange(1, M // 2 + 1)
    return (2.0 / M) * (1.0 - 2.0 * (np.cos(2.0 * np.outer(th, k)) / (4.0 * k ** 2 - 1.0)).sum(axis=1))


@pytest.mark.parametrize("L", [1, 2, 3, 8, 17, 64])
def test_dh_weights_fejer(L):
    assert np.abs(sampling.dh_weights(L) - fejer1(2 * L)).max() < 1e-14


@pytest.mark.parametrize("L", [2, 5, 12])
def test_dh_weights_polynomial_degree(L):
    w, x = sampling.dh_weights(L), np.cos(sampling.thetas_dh(L))
    for k in range(2 * L):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    k = 2 * L   # one degree further the rule is no longer exact
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-12


def test_dh_grid():
    L = 5
    th = sampling.thetas_dh(L)
    assert len(th) == 2 * L == sampling.rings(L, "dh")
    assert abs(th[0] - math.pi / 20) < 1e-15 and abs(th[-1] - 19 * math.pi / 20) < 1e-15
    assert np.all(np.abs(th + th[::-1] - math.pi) < 1e-15)   # symmetric about the equator
    with pytest.raises(ValueError):
        sampling.rings(L, "healpix")


def test_dh_inverse_matches_scipy():
    L = 9
    flm = synth.flm_random(L, synth.rng_for(130, 0))
    T, P = np.meshgrid(sampling.thetas_dh(L), sampling.phis(L), indexing='ij')
    ref = np.zeros_like(T, dtype=complex)
    for l in range(L):
        for m in range(-l, l + 1):
            ref += flm[l, m + L - 1] * ylm_cs(l, m, T, P)
    got = harmonic.sht_inverse(flm, L, 0, samp="dh")
    assert got.shape == (2 * L, 2 * L - 1)
    assert np.abs(got - ref).max() < 1e-13


@pytest.mark.parametrize("spin", [2, -1])
def test_dh_spin_inverse_goldberg(spin):
    L = 5
    th, ph = sampling.thetas_dh(L), sampling.phis(L)
    for l in range(abs(spin), L):
        for m in range(-l, l + 1):
            flm = np.zeros((L, 2 * L - 1), complex)
            flm[l, m + L - 1] = 1.0
            got = harmonic.sht_inverse(flm, L, spin, samp="dh")
            for t in [0, 3, 2 * L - 1]:
                for p in [0, 4]:
                    assert abs(got[t, p] - syl_goldberg(spin, l, m, th[t], ph[p])) < 1e-13


@pytest.mark.parametrize("spin", [0, 1])
def test_dh_forward_single_pixel(spin):
    """Forward DH SHT of one unit pixel: w_t (2 pi/(2L-1)) conj(sY_lm(theta_t, phi_p))."""
    L = 4
    th, ph, w = sampling.thetas_dh(L), sampling.phis(L), sampling.dh_weights(L)
    for (t, p) in [(0, 0), (3, 2), (7, 6)]:
        f = np.zeros((2 * L, 2 * L - 1), complex)
        f[t, p] = 1.0
        got = harmonic.sht_forward(f, L, spin, samp="dh")
        for l in range(abs(spin), L):
            for m in range(-l, l + 1):
                ref = w[t] * (2 * math.pi / (2 * L - 1)) * np.conj(syl_goldberg(spin, l, m, th[t], ph[p]))
                assert abs(got[l, m + L - 1] - ref) < 1e-14


@pytest.mark.parametrize("L,spin", [(1, 0), (2, 0), (8, 0), (16, 0), (8, 2), (7, -1)])
def test_dh_forward_exact_on_bandlimited(L, spin):
    flm = synth.flm_random(L, synth.rng_for(131, L), spin=spin)
    f = harmonic.sht_inverse(flm, L, spin, samp="dh")
    assert np.abs(harmonic.sht_forward(f, L, spin, samp="dh") - flm).max() < 1e-13


def test_dh_forward_agrees_with_mw_route():
    """One band-limited function sampled on both grids has one set of coefficients."""
    L, spin = 10, 2
    flm = synth.flm_random(L, synth.rng_for(132, 0), spin=spin)
    fm = harmonic.sht_inverse(flm, L, spin)
    fd = harmonic.sht_inverse(flm, L, spin, samp="dh")
    a = harmonic.sht_forward(fm, L, spin)
    b = harmonic.sht_forward(fd, L, spin, samp="dh")
    assert np.abs(a - b).max() < 1e-13


def test_dh_wigner_inverse_bruteforce():
    L, N = 4, 3
    flmn = synth.flmn_random(L, N, synth.rng_for(133, 0))
    al, be, ga = sampling.phis(L), sampling.thetas_dh(L), sampling.gammas(N)
    got = harmonic.wigner_inverse(flmn, L, N, samp="dh")
    assert got.shape == (2 * N - 1, 2 * L, 2 * L - 1)
    for g in [0, 4]:
        for b in [0, 5, 2 * L - 1]:
            for a in [0, 3, 6]:
                ref = 0j
                for l in range(L):
                    for m in range(-l, l + 1):
                        for n in range(-min(l, N - 1), min(l, N - 1) + 1):
                            D = d_explicit(l, m, n, be[b]) * np.exp(-1j * (m * al[a] + n * ga[g]))
                            ref += (2 * l + 1) / (8 * math.pi ** 2) * flmn[n + N - 1, l, m + L - 1] * np.conj(D)
                assert abs(got[g, b, a] - ref) < 1e-13


def test_dh_wigner_forward_single_sample():
    """Forward DH Wigner transform of one unit sample: qa qg w_b d^l_mn(beta_b) e^{-i(m a + n g)}."""
    L, N = 3, 2
    al, be, ga, w = sampling.phis(L), sampling.thetas_dh(L), sampling.gammas(N), sampling.dh_weights(L)
    q = (2 * math.pi / (2 * L - 1)) * (2 * math.pi / (2 * N - 1))
    for (g, b, a) in [(0, 0, 0), (2, 4, 3), (1, 5, 1)]:
        f = np.zeros((2 * N - 1, 2 * L, 2 * L - 1), complex)
        f[g, b, a] = 1.0
        got = harmonic.wigner_forward(f, L, N, samp="dh")
        for n in range(-(N - 1), N):
            for l in range(abs(n), L):
                for m in range(-l, l + 1):
                    ref = q * w[b] * d_explicit(l, m, n, be[b]) * np.exp(-1j * (m * al[a] + n * ga[g]))
                    assert abs(got[n + N - 1, l, m + L - 1] - ref) < 1e-14


@pytest.mark.parametrize("L,N", [(1, 1), (3, 2), (8, 3)])
def test_dh_wigner_forward_exact_on_bandlimited(L, N):
    flmn = synth.flmn_random(L, N, synth.rng_for(134, L))
    f = harmonic.wigner_inverse(flmn, L, N, samp="dh")
    assert np.abs(harmonic.wigner_forward(f, L, N, samp="dh") - flmn).max() < 1e-13


def test_dh_wavelet_round_trip_and_mw_agreement():
    """Algorithm 1 on DH: exact round trip on band-limited f, and every wavelet map has the
    Wigner coefficients of the MW analysis of the same function."""
    L, N, lam, J0, spin = 12, 3, 2.0, 1, 2
    flm = synth.flm_random(L, synth.rng_for(135, 0), spin=spin)
    fd = harmonic.sht_inverse(flm, L, spin, samp="dh")
    fm = harmonic.sht_inverse(flm, L, spin)
    wd, pd = wavelet.analysis(fd, L, N, lam, J0, spin, samp="dh")
    wm, pm = wavelet.analysis(fm, L, N, lam, J0, spin)
    for a, b in zip(wd, wm):
        Lj, Nj = a.shape[2] // 2 + 1, a.shape[0] // 2 + 1
        assert a.shape[1] == 2 * Lj
        ca = harmonic.wigner_forward(a, Lj, Nj, samp="dh")
        cb = harmonic.wigner_forward(b, Lj, Nj)
        assert np.abs(ca - cb).max() < 1e-13 * max(1.0, np.abs(cb).max())
    LP = pd.shape[1] // 2 + 1
    assert np.abs(harmonic.sht_forward(pd, LP, 0, samp="dh") - harmonic.sht_forward(pm, LP, 0)).max() < 1e-13
    back = wavelet.synthesis(wd, pd, L, N, lam, J0, spin, samp="dh")
    assert np.abs(back - fd).max() < 1e-12 * np.abs(fd).max()

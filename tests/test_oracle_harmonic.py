"""Pins for the oracle's spin SHT and Wigner transforms (oracle/harmonic.py, sampling.py)."""
import math

import numpy as np
import pytest

import synth
from oracle import harmonic, sampling
from tests.pins import (d_explicit, dirichlet_interp, quad_complex, syl_goldberg, ylm_cs)


def test_sin_weight_closed_form():
    for q in range(-7, 8):
        v = quad_complex(lambda t: np.exp(1j * q * t) * math.sin(t), 0.0, math.pi)
        assert abs(sampling.sin_weight(np.array([q]))[0] - v) < 1e-13


def test_ylm_closed_forms():
    L = 4
    th, ph = sampling.thetas(L), sampling.phis(L)
    T, P = np.meshgrid(th, ph, indexing='ij')
    closed = {
        (0, 0): np.full_like(T, 1 / math.sqrt(4 * math.pi)) + 0j,
        (1, 0): math.sqrt(3 / (4 * math.pi)) * np.cos(T) + 0j,
        (1, 1): -math.sqrt(3 / (8 * math.pi)) * np.sin(T) * np.exp(1j * P),
        (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * np.cos(T) ** 2 - 1) + 0j,
        (2, 2): 0.25 * math.sqrt(15 / (2 * math.pi)) * np.sin(T) ** 2 * np.exp(2j * P),
    }
    for (l, m), ref in closed.items():
        flm = np.zeros((L, 2 * L - 1), complex)
        flm[l, m + L - 1] = 1.0
        assert np.abs(harmonic.sht_inverse(flm, L) - ref).max() < 1e-14


def test_inverse_matches_scipy_synthesis():
    """Spin-0 inverse SHT equals a dense sum of scipy's Condon-Shortley harmonics."""
    L = 9
    flm = synth.flm_random(L, synth.rng_for(100, 0))
    th, ph = sampling.thetas(L), sampling.phis(L)
    T, P = np.meshgrid(th, ph, indexing='ij')
    ref = np.zeros_like(T, dtype=complex)
    for l in range(L):
        for m in range(-l, l + 1):
            ref += flm[l, m + L - 1] * ylm_cs(l, m, T, P)
    assert np.abs(harmonic.sht_inverse(flm, L) - ref).max() < 1e-13


@pytest.mark.parametrize("spin", [1, 2, -1])
def test_spin_harmonics_goldberg(spin):
    """Spin harmonics (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s} e^{im phi} equal Goldberg's explicit formula."""
    L = 5
    th, ph = sampling.thetas(L), sampling.phis(L)
    for l in range(abs(spin), L):
        for m in range(-l, l + 1):
            flm = np.zeros((L, 2 * L - 1), complex)
            flm[l, m + L - 1] = 1.0
            got = harmonic.sht_inverse(flm, L, spin)
            for t in [0, 1, 3]:
                for p in [0, 2, 5]:
                    ref = syl_goldberg(spin, l, m, th[t], ph[p])
                    assert abs(got[t, p] - ref) < 1e-13


@pytest.mark.parametrize("L,spin", [(1, 0), (2, 0), (7, 0), (16, 0), (8, 1), (11, 2), (6, -2)])
def test_forward_exact_on_bandlimited(L, spin):
    flm = synth.flm_random(L, synth.rng_for(101, L), spin=spin)
    f = harmonic.sht_inverse(flm, L, spin)
    assert np.abs(harmonic.sht_forward(f, L, spin) - flm).max() < 1e-13


def _bruteforce_forward(f, L, spin):
    """Forward MW SHT on arbitrary samples: exact phi sums, the unique degree-(L-1)
    trigonometric interpolant of the parity-extended column, then adaptive quadrature of
    int_0^pi G(theta) d^l_{m,-s}(theta) sin(theta) with Wigner's explicit sum."""
    ph = sampling.phis(L)
    out = np.zeros((L, 2 * L - 1), complex)
    for m in range(-(L - 1), L):
        G = (2 * math.pi / (2 * L - 1)) * (f @ np.exp(-1j * m * ph))
        sign = (-1) ** ((m + spin) % 2)
        ext = np.concatenate([G, sign * G[L - 2::-1]]) if L > 1 else G
        g = dirichlet_interp(ext, L)
        for l in range(max(abs(m), abs(spin)), L):
            val = quad_complex(lambda t: g(t) * d_explicit(l, m, -spin, t) * math.sin(t),
                               0.0, math.pi)
            out[l, m + L - 1] = (-1) ** spin * math.sqrt((2 * l + 1) / (4 * math.pi)) * val
    return out


@pytest.mark.parametrize("L,spin", [(3, 0), (4, 1)])
def test_forward_operator_on_arbitrary_samples(L, spin):
    """Pins the whole MW forward operator, including its action off the band-limited subspace."""
    f = synth.pixels_random((L, 2 * L - 1), synth.rng_for(102, L), complex_=True)
    ref = _bruteforce_forward(f, L, spin)
    assert np.abs(harmonic.sht_forward(f, L, spin) - ref).max() < 1e-11


def test_wigner_inverse_bruteforce():
    L, N = 4, 3
    flmn = synth.flmn_random(L, N, synth.rng_for(103, 0))
    al, be, ga = sampling.phis(L), sampling.thetas(L), sampling.gammas(N)
    got = harmonic.wigner_inverse(flmn, L, N)
    for g in range(2 * N - 1):
        for b in range(L):
            for a in [0, 3, 6]:
                ref = 0j
                for l in range(L):
                    for m in range(-l, l + 1):
                        for n in range(-min(l, N - 1), min(l, N - 1) + 1):
                            D = d_explicit(l, m, n, be[b]) * np.exp(-1j * (m * al[a] + n * ga[g]))
                            ref += (2 * l + 1) / (8 * math.pi ** 2) * flmn[n + N - 1, l, m + L - 1] \
                                * np.conj(D)
                assert abs(got[g, b, a] - ref) < 1e-13


def test_wigner_inverse_ring_bruteforce():
    """One ring of Eq. 5 at an arbitrary colatitude (not a grid ring) against Wigner's explicit
    sum for d^l_mn, term by term."""
    L, N, beta = 5, 3, 0.7345
    flmn = synth.flmn_random(L, N, synth.rng_for(104, 0))
    al, ga = sampling.phis(L), sampling.gammas(N)
    got = harmonic.wigner_inverse_ring(flmn, L, N, beta)
    for g in range(2 * N - 1):
        for a in range(2 * L - 1):
            ref = 0j
            for l in range(L):
                for m in range(-l, l + 1):
                    for n in range(-min(l, N - 1), min(l, N - 1) + 1):
                        D = d_explicit(l, m, n, beta) * np.exp(-1j * (m * al[a] + n * ga[g]))
                        ref += (2 * l + 1) / (8 * math.pi ** 2) * flmn[n + N - 1, l, m + L - 1] * np.conj(D)
            assert abs(got[g, a] - ref) < 1e-13


@pytest.mark.parametrize("L,N,samp", [(12, 4, "mw"), (9, 9, "dh"), (16, 2, "mw")])
def test_wigner_inverse_ring_matches_every_ring(L, N, samp):
    """Every grid ring of the full inverse transform, and the pole: at beta = 0, d^l_mn = delta_mn,
    so f(alpha, 0, gamma) = sum_l (2l+1)/(8 pi^2) sum_{|m| < N} f^l_mm exp(i m (alpha + gamma))."""
    flmn = synth.flmn_random(L, N, synth.rng_for(105, L))
    full = harmonic.wigner_inverse(flmn, L, N, samp)
    th = sampling.thetas_for(L, samp)
    scale = np.abs(full).max()
    for t in range(len(th)):
        assert np.abs(harmonic.wigner_inverse_ring(flmn, L, N, th[t]) - full[:, t]).max() < 1e-13 * scale
    al, ga = sampling.phis(L), sampling.gammas(N)
    pole = np.zeros((2 * N - 1, 2 * L - 1), dtype=np.complex128)
    for l in range(L):
        for m in range(-min(l, N - 1), min(l, N - 1) + 1):
            pole += (2 * l + 1) / (8 * math.pi ** 2) * flmn[m + N - 1, l, m + L - 1] * \
                np.exp(1j * m * (al[None, :] + ga[:, None]))
    assert np.abs(harmonic.wigner_inverse_ring(flmn, L, N, 0.0) - pole).max() < 1e-13 * scale


@pytest.mark.parametrize("L,N", [(1, 1), (3, 2), (8, 3), (10, 10)])
def test_wigner_forward_exact_on_bandlimited(L, N):
    flmn = synth.flmn_random(L, N, synth.rng_for(104, L))
    f = harmonic.wigner_inverse(flmn, L, N)
    assert np.abs(harmonic.wigner_forward(f, L, N) - flmn).max() < 1e-13


def test_wigner_forward_operator_on_arbitrary_samples():
    L, N = 3, 2
    f = synth.pixels_random((2 * N - 1, L, 2 * L - 1), synth.rng_for(105, 0), complex_=True)
    al, ga = sampling.phis(L), sampling.gammas(N)
    got = harmonic.wigner_forward(f, L, N)
    for n in range(-(N - 1), N):
        for m in range(-(L - 1), L):
            G = np.einsum('gba,a,g->b', f, np.exp(-1j * m * al), np.exp(-1j * n * ga))
            G *= (2 * math.pi / (2 * L - 1)) * (2 * math.pi / (2 * N - 1))
            sign = (-1) ** ((m + n) % 2)
            g = dirichlet_interp(np.concatenate([G, sign * G[L - 2::-1]]), L)
            for l in range(max(abs(m), abs(n)), L):
                ref = quad_complex(lambda t: g(t) * d_explicit(l, m, n, t) * math.sin(t), 0.0,
                                   math.pi)
                assert abs(got[n + N - 1, l, m + L - 1] - ref) < 1e-11

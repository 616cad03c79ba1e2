"""Pins of oracle.ballwav (directional wavelet transform on the ball, Sec. 3.2, App. A.3-A.4).

* admissibility (Sec. 3.2): (4 pi/(2l+1)) |Phi_l0p|^2 + (8 pi^2/(2l+1)) sum_{j j' n} |Psi^{jj'}_lnp|^2 = 1
  for every l < L, p < P, evaluated from the sphere filters and the radial tiling;
* exact reconstruction: synthesis(analysis(f)) = f for band-limited fields;
* separable reduction: for f(r, w) = K_{p0}(r) g(w) the coefficients factor into the radial
  profile kappa^{j'}(p0) K_{p0}(r_i) on the P_j' rule times the sphere oracle's W^j of g,
  which fixes the radial rule of each scale, the filter products and the index order.
"""
import math

import numpy as np
import pytest

import synth
from oracle import ballwav, filters, harmonic, laguerre, wavelet


@pytest.mark.parametrize("L,P,N,lam,nu,J0,J0r", [(16, 16, 3, 2.0, 2.0, 0, 0), (12, 10, 2, 2.0, 1.7, 1, 2)])
def test_ball_admissibility(L, P, N, lam, nu, J0, J0r):
    phi = ballwav.scaling_filter(L, P, lam, nu, J0, J0r)
    tot = phi ** 2
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        psi = filters.wavelet_filter(L, N, lam, j)
        ang = np.array([(8 * math.pi ** 2 / (2 * l + 1)) * np.sum(np.abs(psi[l]) ** 2) for l in range(L)])
        for (jr, Pj) in ballwav.radial_bandlimits(P, nu, J0r):
            kap = ballwav.radial_kappa(P, nu, jr)
            assert np.all(kap[Pj:] == 0.0)
            tot = tot + np.outer(kap ** 2, ang)
    assert np.abs(tot - 1.0).max() < 1e-13


@pytest.mark.parametrize("L,P,N,J0,J0r,nu", [(8, 8, 2, 0, 0, 2.0), (6, 7, 3, 1, 0, 1.7)])
def test_ball_exact_reconstruction(L, P, N, J0, J0r, nu):
    rng = synth.rng_for(905, L)
    flmp = synth.flmp_random(L, P, rng, reality=True)
    f = laguerre.spherical_laguerre_inverse(flmp, L, P).real
    wavs, wphi = ballwav.analysis(f, L, N, P, 2.0, nu, J0, J0r)
    f2 = ballwav.synthesis(wavs, wphi, L, N, P, 2.0, nu, J0, J0r)
    assert np.abs(f2 - f).max() / np.abs(f).max() < 1e-12


def test_ball_separable_reduction():
    L, P, N, lam, nu, J0, J0r, p0 = 8, 8, 2, 2.0, 2.0, 0, 0, 3
    rng = synth.rng_for(906, L)
    g = harmonic.sht_inverse(synth.flm_random(L, rng, reality=True), L).real
    _, _, Kfull = laguerre.quadrature(P)
    f = np.stack([Kfull[i, p0] * g for i in range(P)])
    wavs, _ = ballwav.analysis(f, L, N, P, lam, nu, J0, J0r)
    wsph, _ = wavelet.analysis(g, L, N, lam, J0, 0, True)
    for si, (j, Lj, Nj) in enumerate(filters.scale_bandlimits(L, N, lam, J0)):
        for (jr, Pj) in ballwav.radial_bandlimits(P, nu, J0r):
            kap = ballwav.radial_kappa(P, nu, jr)[p0]
            _, _, K = laguerre.quadrature(Pj)
            W = wavs[(j, jr)]
            for i in range(Pj):
                prof = kap * K[i, p0] if p0 < Pj else 0.0
                assert np.abs(W[i] - prof * wsph[si]).max() <= 1e-12 * max(1.0, np.abs(wsph[si]).max())

"""Pins of oracle.adjoint (brute-force adjoints of the wavelet transforms, Sec. 4.3).

The adjoint is pinned to things other than its own construction:
* calculus: the gradient of the quadratic loss sum_j mean |W^j|^2 (the differentiation
  study's loss) is 2 A^H W / n; central finite differences of the oracle's own analysis
  must reproduce it along real and imaginary pixel directions (exact for a quadratic up to
  rounding);
* exact reconstruction (Eq. 42 inverts Eqs. 40-41 on band-limited maps): for band-limited x,
  <S^H y, A x> = <y, S A x> = <y, x>;
* the inner-product definition checked against transforms applied directly (not through
  the matrix), which fixes the flattening order and the conjugation.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint, harmonic, wavelet

CASES = [  # L, N, lam, J0, spin, real
    (8, 3, 2.0, 0, 0, True),
    (8, 2, 2.0, 1, 2, False),
    (7, 3, 1.7, 0, 0, True),
]


def inner(u, v):
    return float(np.real(np.vdot(np.asarray(u).ravel(), np.asarray(v).ravel())))


def loss(f, L, N, lam, J0, spin, real):
    wavs, _ = wavelet.analysis(f, L, N, lam, J0, spin, reality=real)
    return sum(float(np.mean(np.abs(w) ** 2)) for w in wavs)


@pytest.mark.parametrize("L,N,lam,J0,spin,real", CASES)
def test_gradient_matches_finite_differences(L, N, lam, J0, spin, real):
    rng = synth.rng_for(900, L)
    f = synth.pixels_random((L, 2 * L - 1), rng, complex_=not real)
    wavs, wphi = wavelet.analysis(f, L, N, lam, J0, spin, reality=real)
    gw = [2.0 * w / w.size for w in wavs]
    grad = adjoint.analysis_adjoint(gw, np.zeros_like(wphi), L, N, lam, J0, spin, reality=real)
    h = 1e-6
    for k in (0, 5, L * (2 * L - 1) // 2, L * (2 * L - 1) - 1):
        t, p = divmod(k, 2 * L - 1)
        dirs = [1.0] if real else [1.0, 1j]
        for d in dirs:
            fp, fm = f.copy(), f.copy()
            fp[t, p] += h * d
            fm[t, p] -= h * d
            fd = (loss(fp, L, N, lam, J0, spin, real) - loss(fm, L, N, lam, J0, spin, real)) / (2 * h)
            an = grad[t, p].real if d == 1.0 else grad[t, p].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, np.abs(grad).max()), (k, d, fd, an)


@pytest.mark.parametrize("L,N,lam,J0,spin,real", CASES)
def test_synthesis_adjoint_by_exact_reconstruction(L, N, lam, J0, spin, real):
    rng = synth.rng_for(901, L)
    a = synth.flm_random(L, rng, spin=spin, reality=real)
    x = harmonic.sht_inverse(a, L, spin)
    x = x.real if real else x
    y = synth.pixels_random((L, 2 * L - 1), rng, complex_=not real)
    gw, gphi = adjoint.synthesis_adjoint(y, L, N, lam, J0, spin, reality=real)
    wavs, wphi = wavelet.analysis(x, L, N, lam, J0, spin, reality=real)
    lhs = sum(inner(g, w) for g, w in zip(gw, wavs)) + inner(gphi, wphi)
    assert abs(lhs - inner(y, x)) <= 1e-12 * np.linalg.norm(y) * np.linalg.norm(x)


@pytest.mark.parametrize("L,N,lam,J0,spin,real", CASES[:2])
def test_inner_product_definition(L, N, lam, J0, spin, real):
    rng = synth.rng_for(902, L)
    x = synth.pixels_random((L, 2 * L - 1), rng, complex_=not real)
    wavs, wphi = wavelet.analysis(x, L, N, lam, J0, spin, reality=real)
    gw = [synth.pixels_random(w.shape, rng, complex_=not real) for w in wavs]
    gphi = synth.pixels_random(wphi.shape, rng, complex_=not real)
    gx = adjoint.analysis_adjoint(gw, gphi, L, N, lam, J0, spin, reality=real)
    lhs = sum(inner(g, w) for g, w in zip(gw, wavs)) + inner(gphi, wphi)
    assert abs(lhs - inner(gx, x)) <= 1e-12 * (np.linalg.norm(np.concatenate([g.ravel() for g in gw])) + 1) * np.linalg.norm(x)
    # synthesis side, applied directly
    f2 = wavelet.synthesis(gw, gphi, L, N, lam, J0, spin, reality=real)
    gw2, gphi2 = adjoint.synthesis_adjoint(x, L, N, lam, J0, spin, reality=real)
    lhs = sum(inner(g, w) for g, w in zip(gw2, gw)) + inner(gphi2, gphi)
    assert abs(lhs - inner(x, f2)) <= 1e-12 * np.linalg.norm(x) * (np.linalg.norm(f2) + 1) * 10

"""Pins for the oracle's wavelet dictionary (oracle/filters.py)."""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import filters

CASES = [(32, 4, 2.0, 0), (256, 8, 2.0, 2), (64, 5, 1.7, 1), (20, 1, 3.0, 1), (17, 2, 2.0, 3)]


@pytest.mark.parametrize("L,N,lam,J0", CASES)
def test_admissibility(L, N, lam, J0):
    """Eq. 30: (4 pi/(2l+1)) |Phi_l0|^2 + (8 pi^2/(2l+1)) sum_j sum_m |Psi^j_lm|^2 = 1 for all l."""
    phi = filters.scaling_filter(L, lam, J0)
    tot = np.array([4 * math.pi / (2 * l + 1) * phi[l] ** 2 for l in range(L)])
    for (j, Lj, Nj) in filters.scale_bandlimits(L, N, lam, J0):
        psi = filters.wavelet_filter(L, N, lam, j)
        assert np.all(psi[Lj:] == 0)                       # band-limit L_j covers the support
        assert np.all(psi[:, :N - Nj] == 0) and np.all(psi[:, N + Nj - 1:] == 0)
        tot += np.array([8 * math.pi ** 2 / (2 * l + 1) * np.sum(np.abs(psi[l]) ** 2)
                         for l in range(L)])
    assert np.abs(tot - 1).max() < 2e-15


@pytest.mark.parametrize("lam", [2.0, 1.7, 3.0])
def test_support_intervals(lam):
    """Eq. 38: scale j is non-zero only for l in (lambda^(j-1), lambda^(j+1)); Phi only below lambda^J0."""
    for j in range(0, 6):
        for l in range(0, int(lam ** (j + 1)) + 3):
            k = filters.kappa_lambda(l / lam ** j, lam)
            inside = lam ** (j - 1) < l < lam ** (j + 1)
            assert (k > 0) == inside or (inside and k < 1e-300)
    for J0 in range(0, 4):
        phi = filters.scaling_filter(40, lam, J0)
        for l in range(40):
            assert (phi[l] > 0) == (l < lam ** J0)


def test_zeta_partition_and_reality():
    for N in range(1, 9):
        for l in range(1, 20):
            z = np.array([filters.zeta(l, m, N) for m in range(-l, l + 1)])
            assert abs(np.sum(np.abs(z) ** 2) - 1) < 1e-15       # sum_m |zeta_lm|^2 = 1
            assert np.count_nonzero(z) == min(N, l + 1 if (N + l) % 2 else l)
            for m in range(-l, l + 1):                           # zeta_{l,-m} = (-1)^m conj zeta_lm
                assert abs(filters.zeta(l, -m, N) - (-1) ** m * np.conj(filters.zeta(l, m, N))) < 1e-16
        assert filters.zeta(0, 0, N) == (1.0 if N % 2 == 1 else 0.0)


def test_k_lambda_against_tanh_sinh():
    """k_lambda (Eq. A4) from QUADPACK agrees with 30-digit tanh-sinh quadrature."""
    lam = 2.0
    with mp.workdps(30):
        def s(u):
            return mp.exp(-1 / (1 - u * u)) if -1 < u < 1 else mp.mpf(0)

        def f(u):
            return s(2 * lam / (lam - 1) * (u - 1 / lam) - 1) ** 2 / u
        norm = mp.quad(f, [1 / lam, 0.75, 1])
        for t in [0.52, 0.61, 0.75, 0.9, 0.98]:
            ref = float(mp.quad(f, [t, 1]) / norm)
            assert abs(filters.k_lambda(t, lam) - ref) < 3e-16
    assert filters.k_lambda(0.5, lam) == 1.0 and filters.k_lambda(1.0, lam) == 0.0


def test_scales():
    assert filters.scale_bandlimits(256, 8, 2.0, 2) == [(2, 8, 8), (3, 16, 8), (4, 32, 8), (5, 64, 8),
                                                        (6, 128, 8), (7, 256, 8), (8, 256, 8)]
    assert filters.scaling_bandlimit(256, 2.0, 2) == 4
    assert filters.scale_bandlimits(32, 4, 2.0, 0)[0] == (0, 2, 2)


def test_kappa_near_support_edges():
    """kappa^2 keeps full relative precision at the support edges (30-digit tanh-sinh pin),
    where k(t/lambda) - k(t) as a difference of two numbers near 1 would round to 0."""
    lam = 2.0
    with mp.workdps(30):
        def s(u):
            return mp.exp(-1 / (1 - u * u)) if -1 < u < 1 else mp.mpf(0)

        def f(u):
            return s(2 * lam / (lam - 1) * (u - 1 / lam) - 1) ** 2 / u
        norm = mp.quad(f, [1 / lam, 0.75, 1])
        for l in [65, 66, 70, 100, 250, 255]:
            t = l / 128.0
            ref = float(mp.sqrt(mp.quad(f, [max(t / lam, 1 / lam), min(t, 1)]) / norm))
            got = filters.kappa_lambda(t, lam)
            # relative 1e-14, with an absolute floor far below what any output can resolve
            assert abs(got - ref) <= 1e-14 * ref + 1e-18, (l, got, ref)

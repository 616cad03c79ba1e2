"""Pins for the oracle's Fourier-Laguerre transform (oracle/laguerre.py)."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import eval_genlaguerre, roots_genlaguerre

import synth
from oracle import harmonic, laguerre


def K_scipy(p, r, tau):
    return math.sqrt(math.factorial(p) / math.factorial(p + 2)) * math.exp(-r / (2 * tau)) * \
        tau ** -1.5 * eval_genlaguerre(p, 2, r / tau)


@pytest.mark.parametrize("P", [4, 12, 24])
def test_nodes_against_scipy(P):
    r, om, K = laguerre.quadrature(P, 1.0)
    x, _ = roots_genlaguerre(P, 2)
    assert np.abs(r - x).max() < 1e-11 * x.max()


def test_closed_forms_and_basis():
    tau = 1.3
    r, om, K = laguerre.quadrature(6, tau)
    for i in range(6):
        x = r[i] / tau
        assert abs(eval_genlaguerre(1, 2, x) - (3 - x)) < 1e-12 * max(1, x)
        for p in range(6):
            assert abs(K[i, p] - K_scipy(p, r[i], tau)) < 1e-13 * max(1.0, abs(K[i, p]))


def test_orthonormality_by_adaptive_quadrature():
    """int_0^inf K_p K_p' r^2 dr = delta_pp' (Eq. 6-8), with scipy's Laguerre polynomials."""
    tau = 0.8
    for p in range(5):
        for q in range(5):
            v, _ = integrate.quad(lambda r: K_scipy(p, r, tau) * K_scipy(q, r, tau) * r * r, 0, np.inf,
                                  limit=200)
            assert abs(v - (1.0 if p == q else 0.0)) < 1e-10


@pytest.mark.parametrize("P,tau", [(8, 1.0), (32, 0.5), (128, 1.0)])
def test_quadrature_exactness(P, tau):
    r, om, K = laguerre.quadrature(P, tau)
    assert np.abs((K * om[:, None]).T @ K - np.eye(P)).max() < 1e-12
    c = np.random.default_rng(P).normal(size=(P, 3))
    assert np.abs(laguerre.radial_forward(laguerre.radial_inverse(c, P, tau), P, tau) - c).max() < 1e-12


def test_single_basis_function():
    P, tau = 10, 1.0
    r, _, _ = laguerre.quadrature(P, tau)
    f = np.array([K_scipy(3, x, tau) for x in r])
    fp = laguerre.radial_forward(f, P, tau)
    assert np.abs(fp - np.eye(P)[3]).max() < 1e-13


def test_spherical_laguerre_round_trip():
    L, P = 8, 6
    flmp = synth.flmp_random(L, P, synth.rng_for(300, 0))
    f = laguerre.spherical_laguerre_inverse(flmp, L, P).real
    assert np.abs(laguerre.spherical_laguerre_forward(f, L, P) - flmp).max() < 1e-13

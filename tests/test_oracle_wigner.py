"""Pins for the oracle's Wigner-d functions (oracle/wigner.py)."""
import math

import numpy as np
import pytest

from oracle import wigner
from tests.pins import d_explicit, quad_complex

BETAS = [0.0, 0.3, 1.1, math.pi / 2, 2.4, math.pi - 1e-3, math.pi]


@pytest.mark.parametrize("beta", BETAS)
def test_closed_forms_l1_l2(beta):
    c, s = math.cos(beta), math.sin(beta)
    d1 = wigner.d_matrix(1, beta)
    d2 = wigner.d_matrix(2, beta)
    ref1 = {(1, 1): (1 + c) / 2, (1, 0): -s / math.sqrt(2), (1, -1): (1 - c) / 2, (0, 0): c}
    ref2 = {(2, 2): ((1 + c) / 2) ** 2, (2, 1): -(1 + c) * s / 2, (2, 0): math.sqrt(3 / 8) * s * s,
            (2, -1): -(1 - c) * s / 2, (2, -2): ((1 - c) / 2) ** 2, (1, 1): (1 + c) * (2 * c - 1) / 2,
            (1, 0): -math.sqrt(1.5) * s * c, (1, -1): (1 - c) * (2 * c + 1) / 2,
            (0, 0): (3 * c * c - 1) / 2}
    for (m, n), v in ref1.items():
        assert abs(d1[m + 1, n + 1] - v) < 2e-15
    for (m, n), v in ref2.items():
        assert abs(d2[m + 2, n + 2] - v) < 2e-15


@pytest.mark.parametrize("l", [3, 7, 12])
def test_explicit_sum(l):
    rng = np.random.default_rng(l)
    for beta in [0.17, 1.3, 2.9]:
        D = wigner.d_matrix(l, beta)
        for _ in range(25):
            m, n = rng.integers(-l, l + 1, size=2)
            assert abs(D[m + l, n + l] - d_explicit(l, int(m), int(n), beta)) < 5e-15


def test_symmetries_and_unitarity():
    l = 40
    D = wigner.d_matrix(l, 0.83)
    m = np.arange(-l, l + 1)
    sign = (-1.0) ** ((m[:, None] - m[None, :]) % 2)
    assert np.abs(D[::-1, ::-1] - sign * D).max() < 1e-14          # d_{-m,-n} = (-1)^(m-n) d_mn
    assert np.abs(D.T - sign * D).max() < 1e-14                     # d_nm = (-1)^(m-n) d_mn
    assert np.abs(D @ D.T - np.eye(2 * l + 1)).max() < 1e-13        # unitarity


def test_group_property():
    """d^l(b1 + b2) = d^l(b1) d^l(b2): rotations about one axis compose."""
    for l in [5, 30, 64]:
        a, b = 0.61, 1.37
        lhs = wigner.d_matrix(l, a + b)
        rhs = wigner.d_matrix(l, a) @ wigner.d_matrix(l, b)
        assert np.abs(lhs - rhs).max() < 5e-13


@pytest.mark.parametrize("lmn", [(3, 5, 1, 0), (4, 4, 2, -1), (6, 9, 3, 3), (10, 10, -7, 2)])
def test_orthogonality(lmn):
    """int_0^pi d^l_mn d^l'_mn sin(beta) d beta = 2/(2l+1) delta_ll' (adaptive quadrature)."""
    l1, l2, m, n = lmn
    v = quad_complex(lambda b: wigner.d_values(l1, m, n, np.array([b]))[0] *
                     wigner.d_values(l2, m, n, np.array([b]))[0] * math.sin(b) + 0j, 0.0, math.pi)
    expect = 2.0 / (2 * l1 + 1) if l1 == l2 else 0.0
    assert abs(v - expect) < 1e-12


def test_fourier_coeff_degree():
    """c^l_mn(k) vanishes for |k| > l by construction and d is real."""
    C = wigner.fourier_coeffs(9)
    k = np.arange(-9, 10)
    val = C @ np.exp(1j * k * 0.77)
    assert np.abs(val.imag).max() < 1e-14

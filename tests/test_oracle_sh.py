"""Pins for the oracle's SH basis (Sec. 4.2, Eq. 6): the recursion-built
real basis against the textbook Cartesian table, orthonormality under an
exact quadrature, and the addition theorem."""
import math

import numpy as np
import pytest

import oracle
from tests.trees import cartesian_table

pytestmark = pytest.mark.filterwarnings("ignore")


def test_dc_constant():
    for d in [(0, 0, 1), (1, 0, 0), (0.3, -0.4, 0.5)]:
        assert oracle.sh_basis(0, d)[0] == pytest.approx(1 / (2 * math.sqrt(math.pi)), abs=1e-16)


def test_matches_cartesian_table():
    rng = np.random.default_rng(0)
    for _ in range(200):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        got = oracle.sh_basis(4, v)
        np.testing.assert_allclose(got, cartesian_table(*v), rtol=0, atol=4e-15)
        np.testing.assert_array_equal(oracle.sh_basis(3, v), got[:16])


def test_signs_and_index_order():
    c1 = math.sqrt(3 / (4 * math.pi))
    assert oracle.sh_basis(1, (1, 0, 0))[3] == pytest.approx(c1)   # m=+1 ~ x
    assert oracle.sh_basis(1, (0, 1, 0))[1] == pytest.approx(c1)   # m=-1 ~ y
    assert oracle.sh_basis(1, (0, 0, 1))[2] == pytest.approx(c1)   # m=0 ~ z
    # m < 0 terms are sin(|m| phi): they vanish on the xz half-plane phi = 0
    Y = oracle.sh_basis(4, (0.6, 0.0, 0.8))
    for l in range(1, 5):
        for m in range(-l, 0):
            assert abs(Y[l * (l + 1) + m]) < 1e-15


def test_orthonormal_under_exact_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi is exact for the products
    # Y_i Y_j of degree <= 8.
    deg = 4
    K = (deg + 1) ** 2
    xs, ws = np.polynomial.legendre.leggauss(8)
    nphi = 20
    G = np.zeros((K, K))
    for z, w in zip(xs, ws):
        s = math.sqrt(1 - z * z)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            Y = oracle.sh_basis(deg, (s * math.cos(ph), s * math.sin(ph), z))
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(K), atol=1e-13)


def test_addition_theorem():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b = rng.normal(size=3), rng.normal(size=3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ya, Yb = oracle.sh_basis(4, a), oracle.sh_basis(4, b)
        for l in range(5):
            sl = slice(l * l, (l + 1) ** 2)
            lhs = float(np.dot(Ya[sl], Yb[sl]))
            rhs = (2 * l + 1) / (4 * math.pi) * np.polynomial.legendre.Legendre.basis(l)(float(np.dot(a, b)))
            assert lhs == pytest.approx(rhs, abs=1e-14)


def test_direction_is_normalised():
    np.testing.assert_allclose(oracle.sh_basis(3, (2.0, -1.0, 0.5)),
                               oracle.sh_basis(3, np.array([2.0, -1.0, 0.5]) / math.sqrt(5.25)), atol=1e-15)

"""Pins for the oracle's 1D rules and Lagrange basis (Section 1: Q_p on Gauss-Lobatto points)."""
import math
import os

import numpy as np
import pytest

from oracle.quadrature import gauss, gll, lagrange, legendre

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_closed_forms.txt")


def _closed_forms():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, xs, ws = [s.strip() for s in line.split("|")]
        kind, n = head.split()
        ev = lambda s: [eval(t, {"sqrt": math.sqrt}) for t in s.split(",")]
        rows.append((kind, int(n), ev(xs), ev(ws)))
    return rows


@pytest.mark.parametrize("kind,n,xs,ws", _closed_forms())
def test_closed_forms(kind, n, xs, ws):
    x, w = (gll if kind == "gll" else gauss)(n)
    np.testing.assert_allclose(x, xs, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, ws, rtol=0, atol=4e-16)


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_matches_library(n):
    x, w = gauss(n)
    xl, wl = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xl, atol=1e-15)
    np.testing.assert_allclose(w, wl, atol=1e-14)


def _moment(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("n", range(2, 11))
def test_exactness_degrees(n):
    # Gauss with n points is exact to degree 2n-1, GLL to 2n-3, and neither to the next even degree
    x, w = gauss(n)
    for k in range(2 * n):
        assert abs(w @ x ** k - _moment(k)) < 1e-13
    assert abs(w @ x ** (2 * n) - _moment(2 * n)) > 1e-6
    x, w = gll(n)
    for k in range(2 * n - 2):
        assert abs(w @ x ** k - _moment(k)) < 1e-13
    assert abs(w @ x ** (2 * n - 2) - _moment(2 * n - 2)) > 1e-6


def test_legendre_values():
    # P_2 = (3x^2-1)/2, P_3 = (5x^3-3x)/2 and derivatives
    x = np.linspace(-1, 1, 7)
    p, d, s = legendre(3, x)
    np.testing.assert_allclose(p, (5 * x ** 3 - 3 * x) / 2, atol=1e-15)
    np.testing.assert_allclose(d, (15 * x ** 2 - 3) / 2, atol=1e-14)
    np.testing.assert_allclose(s, 15 * x, atol=1e-13)
    p, d, _ = legendre(2, x)
    np.testing.assert_allclose(p, (3 * x ** 2 - 1) / 2, atol=1e-15)


@pytest.mark.parametrize("P", range(2, 10))
def test_lagrange_basis(P):
    nodes, _ = gll(P)
    L, dL = lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(P), atol=1e-14)
    rng = np.random.default_rng(P)
    x = rng.uniform(-1, 1, 11)
    L, dL = lagrange(nodes, x)
    np.testing.assert_allclose(L.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dL.sum(1), 0.0, atol=1e-11)
    # interpolation of monomials of degree <= p is exact, and so is their derivative
    for m in range(P):
        np.testing.assert_allclose(L @ nodes ** m, x ** m, atol=1e-12)
        np.testing.assert_allclose(dL @ nodes ** m, m * x ** max(m - 1, 0) if m else 0 * x, atol=1e-10)
    # derivative against a central difference of the values
    h = 1e-6
    Lp, _ = lagrange(nodes, x + h)
    Lm, _ = lagrange(nodes, x - h)
    np.testing.assert_allclose(dL, (Lp - Lm) / (2 * h), atol=1e-6 * P ** 2)


@pytest.mark.parametrize("P", range(2, 10))
def test_gll_derivative_matrix(P):
    # D_ij = l_j'(x_i) on GLL nodes: corner entries -+ p(p+1)/4 and centro-antisymmetry
    p = P - 1
    nodes, _ = gll(P)
    _, D = lagrange(nodes, nodes)
    assert abs(D[0, 0] + p * (p + 1) / 4) < 1e-12
    assert abs(D[-1, -1] - p * (p + 1) / 4) < 1e-12
    np.testing.assert_allclose(D, -D[::-1, ::-1], atol=1e-12)

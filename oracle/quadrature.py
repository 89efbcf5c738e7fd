"""1D quadrature rules and Lagrange bases for the oracle (test infrastructure).

The paper builds Q_p elements on Lagrange polynomials through the
Gauss-Lobatto points (Section 1, "Let Q_p denote the Lagrange polynomial bases
on Gauss-Lobatto quadrature points") and integrates either at the same points
(collocated quadrature, BP5) or at Gauss points (BP1/BP3).  The rules here are
the textbook ones, computed with a Newton iteration on Legendre polynomials
evaluated by Bonnet's three-term recurrence:

  Gauss, n points:        roots of P_n,                 w = 2 / ((1 - x^2) P_n'(x)^2)
  Gauss-Lobatto, n points: +-1 and the roots of P_{n-1}', w = 2 / (n (n-1) P_{n-1}(x)^2)
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """(P_n(x), P_n'(x), P_n''(x)) by Bonnet's recurrence; x may be an array."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    s0, s1 = np.zeros_like(x), np.zeros_like(x)
    if n == 0:
        return p0, d0, s0
    for k in range(1, n):
        # (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; differentiate it once and twice
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = ((2 * k + 1) * (p1 + x * d1) - k * d0) / (k + 1)
        s2 = ((2 * k + 1) * (2 * d1 + x * s1) - k * s0) / (k + 1)
        p0, p1, d0, d1, s0, s1 = p1, p2, d1, d2, s1, s2
    return p1, d1, s1


def gauss(n: int):
    """n-point Gauss-Legendre nodes (ascending) and weights."""
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n)
    x = -np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp, _ = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp, _ = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gll(n: int):
    """n-point Gauss-Lobatto-Legendre nodes (ascending, including +-1) and weights."""
    if n < 2:
        raise ValueError("n >= 2")
    m = n - 1
    x = -np.cos(np.pi * np.arange(n) / m)
    if n > 2:
        xi = x[1:-1].copy()
        for _ in range(100):
            p, dp, d2p = legendre(m, xi)
            dx = dp / d2p
            xi = xi - dx
            if np.max(np.abs(dx)) < 1e-16:
                break
        x[1:-1] = xi
    x[0], x[-1] = -1.0, 1.0
    p, _, _ = legendre(m, x)
    w = 2.0 / (n * m * p * p)
    return x, w


def lagrange(nodes, x):
    """Values L[k, j] = l_j(x_k) and derivatives dL[k, j] = l_j'(x_k).

    l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m); its derivative is the sum
    over l != j of the same product with the factor for l replaced by
    1 / (x_j - x_l).  Written out term by term: O(n^3) per point.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
        for l in range(n):
            if l == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[l]))
            for m in range(n):
                if m != j and m != l:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            dL[:, j] += term
    return L, dL


def rule(kind: str, n: int):
    """Quadrature rule by name: 'gll' or 'gauss' with n points."""
    if kind == "gll":
        return gll(n)
    if kind == "gauss":
        return gauss(n)
    raise ValueError(f"unknown rule {kind}")

"""Pins for the oracle's non-tensor (tetrahedral) elements.

Independent checks: the conical rule integrates monomials exactly against the closed form
int_T x^a y^b z^c = a! b! c! / (a+b+c+3)! up to degree 2q - 1 (and not beyond); the Silvester
basis is cardinal at the nodes, reproduces P_p and its gradients, matches finite differences,
and its element matrices equal those of the exact rational Vandermonde inverse integrated
monomial by monomial (a second, exact construction of the same basis); the P1 element matrices
on the reference tetrahedron have their textbook closed forms; on the Kuhn mesh shared nodes
coincide physically, 1^T M 1 = |Omega| = 1, A 1 = 0, A is symmetric and positive semidefinite, the
linear patch test holds, dense action = assembled matrix, and the manufactured solution converges
at O(h^{p+1}).
"""
from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem
from oracle import simplex as sx


def _monomials(deg):
    return [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)]


def _exact_monomial(a, b, c):
    return factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_conical_rule_exactness(q):
    XI, W = sx.conical_rule(q)
    assert XI.shape == (q ** 3, 3)
    assert (XI > 0).all() and (XI.sum(1) < 1).all()
    assert abs(W.sum() - 1.0 / 6.0) < 1e-15
    for a, b, c in _monomials(2 * q - 1):
        val = (W * XI[:, 0] ** a * XI[:, 1] ** b * XI[:, 2] ** c).sum()
        assert abs(val - _exact_monomial(a, b, c)) <= 1e-15 * max(1.0, _exact_monomial(a, b, c)) * 10, (a, b, c)
    # one degree higher is not integrated exactly by the collapsed u-direction
    val = (W * XI[:, 0] ** (2 * q)).sum()
    assert abs(val - _exact_monomial(2 * q, 0, 0)) > 1e-12 * _exact_monomial(2 * q, 0, 0)


def test_one_point_rule_closed_form():
    # q = 1: the single point is the centroid (1/4, 1/4, 1/4) with weight |T| = 1/6
    XI, W = sx.conical_rule(1)
    np.testing.assert_allclose(XI[0], [0.25, 0.25, 0.25], atol=1e-15)
    np.testing.assert_allclose(W, [1.0 / 6.0], atol=1e-16)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_basis_cardinal_and_reproducing(p):
    N = sx.nodes(p)
    assert N.shape[0] == sx.n_nodes(p)
    np.testing.assert_array_equal(sx.multi_indices(p), synthetic.simplex_multi_indices(p))
    Phi, _ = sx.basis(p, N)
    np.testing.assert_allclose(Phi, np.eye(len(N)), atol=1e-13)
    rng = np.random.default_rng(p)
    pts = rng.dirichlet(np.ones(4), size=40)[:, 1:]
    Phi, dPhi = sx.basis(p, pts)
    for a, b, c in _monomials(p):
        f = N[:, 0] ** a * N[:, 1] ** b * N[:, 2] ** c
        ref = pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c
        np.testing.assert_allclose(Phi @ f, ref, atol=1e-12)
        grads = [a * pts[:, 0] ** max(a - 1, 0) * pts[:, 1] ** b * pts[:, 2] ** c,
                 b * pts[:, 0] ** a * pts[:, 1] ** max(b - 1, 0) * pts[:, 2] ** c,
                 c * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** max(c - 1, 0)]
        for d in range(3):
            np.testing.assert_allclose(dPhi[d] @ f, grads[d], atol=1e-10)


@pytest.mark.parametrize("p", [2, 4])
def test_basis_gradient_finite_differences(p):
    rng = np.random.default_rng(10 + p)
    pts = rng.dirichlet(np.ones(4), size=10)[:, 1:] * 0.9 + 0.025
    _, dPhi = sx.basis(p, pts)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (sx.basis(p, pts + e)[0] - sx.basis(p, pts - e)[0]) / (2 * h)
        np.testing.assert_allclose(dPhi[d], fd, atol=1e-7)


def _exact_basis_coefficients(p):
    """Monomial coefficients of the Lagrange basis by exact (rational) inversion of the Vandermonde
    matrix at the equispaced nodes: C[m][n], phi_n = sum_m C[m][n] x^a y^b z^c."""
    mons = _monomials(p)
    nodes = [tuple(Fraction(int(v), p) for v in row) for row in sx.multi_indices(p)]
    n = len(nodes)
    V = [[nd_[0] ** a * nd_[1] ** b * nd_[2] ** c for (a, b, c) in mons] for nd_ in nodes]
    # Gauss-Jordan on [V | I] in exact arithmetic: V C = I
    M = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(V)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [vr - f * vc for vr, vc in zip(M[r], M[col])]
    C = [[M[m][n + j] for j in range(n)] for m in range(n)]
    return mons, C


@pytest.mark.parametrize("p", [2, 3])
def test_element_matrices_equal_exact_rational_construction(p):
    # reference tetrahedron, k = rho = 1: mass and stiffness by the oracle's quadrature against
    # the exact monomial expansion of the basis integrated with the closed-form monomial integrals
    mons, C = _exact_basis_coefficients(p)
    n = len(mons)

    def mono_int(a, b, c):
        return Fraction(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))

    Mm = [[mono_int(a1 + a2, b1 + b2, c1 + c2) for (a2, b2, c2) in mons] for (a1, b1, c1) in mons]
    Km = [[Fraction(0)] * n for _ in range(n)]
    for i, (a1, b1, c1) in enumerate(mons):
        for j, (a2, b2, c2) in enumerate(mons):
            s = Fraction(0)
            for (e1, e2) in ((a1 * a2, (a1 + a2 - 2, b1 + b2, c1 + c2)), (b1 * b2, (a1 + a2, b1 + b2 - 2, c1 + c2)),
                             (c1 * c2, (a1 + a2, b1 + b2, c1 + c2 - 2))):
                if e1:
                    s += e1 * mono_int(*e2)
            Km[i][j] = s
    Mex = np.array([[float(sum(C[a][i] * Mm[a][b] * C[b][j] for a in range(n) for b in range(n)))
                     for j in range(n)] for i in range(n)])
    Kex = np.array([[float(sum(C[a][i] * Km[a][b] * C[b][j] for a in range(n) for b in range(n)))
                     for j in range(n)] for i in range(n)])
    ref_tet = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=np.float64)
    sp_ = sx.SimplexSpace(p, p + 1)
    M = fem.element_matrices(sp_, sx.qdata_mass(sp_, ref_tet), fem.MASS)[0]
    K = fem.element_matrices(sp_, sx.qdata_diffusion(sp_, ref_tet), fem.DIFFUSION)[0]
    np.testing.assert_allclose(M, Mex, atol=1e-15)
    np.testing.assert_allclose(K, Kex, atol=1e-13)


def test_p1_reference_matrices_closed_form():
    ref_tet = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=np.float64)
    sp_ = sx.SimplexSpace(1, 2)
    M = fem.element_matrices(sp_, sx.qdata_mass(sp_, ref_tet), fem.MASS)[0]
    K = fem.element_matrices(sp_, sx.qdata_diffusion(sp_, ref_tet), fem.DIFFUSION)[0]
    np.testing.assert_allclose(M, (np.ones((4, 4)) + np.eye(4)) / 120.0, atol=1e-16)
    Kref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    np.testing.assert_allclose(K, Kref, atol=1e-15)


def test_kuhn_mesh_conforming_and_positive():
    for p in (1, 2, 3):
        m = synthetic.TetMesh(3, 2, 2, p, seed=5)
        assert m.n_ldof == (3 * p + 1) * (2 * p + 1) ** 2
        assert np.unique(m.elem_dofs).size == m.n_ldof
        _, J = sx.affine_map(m.vertices, np.zeros((1, 3)))
        assert np.linalg.det(J).min() > 0
        X = sx.node_points(p, m.vertices)                      # [E, nd, 3] per element
        ref = np.full((m.n_ldof, 3), np.nan)
        ref[m.elem_dofs.reshape(-1)] = X.reshape(-1, 3)
        np.testing.assert_allclose(X, ref[m.elem_dofs], atol=1e-15)   # every element agrees on shared nodes
        # boundary nodes are exactly the nodes on the boundary of the (fixed) unit cube
        onb = ((ref < 1e-14) | (ref > 1 - 1e-14)).any(1)
        np.testing.assert_array_equal(onb, m.boundary.astype(bool))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_total_volume_and_diffusion_kernel(p):
    m = synthetic.TetMesh(2, 2, 3, p, seed=2)
    sp_ = sx.SimplexSpace(p, p + 1)
    one = np.ones(m.n_ldof)
    M1 = fem.apply(sp_, m.elem_dofs, sx.qdata_mass(sp_, m.vertices), one, fem.MASS)
    assert abs(one @ M1 - 1.0) < 1e-13
    y = fem.apply(sp_, m.elem_dofs, sx.qdata_diffusion(sp_, m.vertices, "sine"), one, fem.DIFFUSION)
    assert np.abs(y).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetric_psd_and_assembled(p):
    m = synthetic.TetMesh(2, 1, 1, p, seed=4)
    sp_ = sx.SimplexSpace(p, p + 1)
    for op, qd in ((fem.MASS, sx.qdata_mass(sp_, m.vertices)),
                   (fem.DIFFUSION, sx.qdata_diffusion(sp_, m.vertices, "sine"))):
        A = fem.assemble(sp_, m.elem_dofs, qd, op, m.n_ldof).toarray()
        np.testing.assert_allclose(A, A.T, atol=1e-14)
        ev = np.linalg.eigvalsh(A)
        assert ev.min() > -1e-12 * ev.max()
        x = synthetic.uniform(m.n_ldof, seed=3)
        np.testing.assert_allclose(fem.apply(sp_, m.elem_dofs, qd, x, op), A @ x, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_linear_patch_test(p):
    # u = c . x lies in P_p on every (affine) element: (A u)_i = 0 at interior nodes for k = 1
    m = synthetic.TetMesh(3, 3, 2, p, seed=6)
    sp_ = sx.SimplexSpace(p, p)
    X = sx.node_points(p, m.vertices)
    xyz = np.zeros((m.n_ldof, 3))
    xyz[m.elem_dofs.reshape(-1)] = X.reshape(-1, 3)
    u = xyz @ np.array([0.4, -0.9, 1.3])
    y = fem.apply(sp_, m.elem_dofs, sx.qdata_diffusion(sp_, m.vertices), u, fem.DIFFUSION)
    inner = ~m.boundary.astype(bool)
    assert np.abs(y[inner]).max() < 1e-12 * np.abs(y).max()
    assert np.abs(y[~inner]).max() > 1e-3


def _solve(N, p):
    m = synthetic.TetMesh(N, N, N, p, seed=0)
    sp_ = sx.SimplexSpace(p, p + 1)
    G = sx.qdata_diffusion(sp_, m.vertices, "sine")
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).tolil()
    mask = m.boundary.astype(bool)
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    b = sx.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    u = spla.spsolve(A.tocsc(), b)
    return sx.l2_error(p, m.vertices, m.elem_dofs, u)


@pytest.mark.parametrize("p,Ns", [(1, (4, 8)), (2, (3, 6)), (3, (2, 4))])
def test_convergence_order(p, Ns):
    e = [_solve(N, p) for N in Ns]
    rate = np.log(e[0] / e[1]) / np.log(Ns[1] / Ns[0])
    assert p + 0.7 <= rate <= p + 1.6, (e, rate)

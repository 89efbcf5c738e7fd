"""Pins for the oracle's conforming hp (variable order) spaces.

Independent checks: with one order everywhere the space and operator are the standard ones (up to
the documented true-dof numbering); for random orders per element the field P x is continuous
across every interior face (both elements' polynomials agree at random face points), polynomials
of degree <= the lowest order are reproduced exactly, linear functions are in the space under the
trilinear maps (linear patch test), the operator is symmetric positive semidefinite with A 1 = 0,
1^T M 1 = |Omega|, and the manufactured solution converges at the rate of the lowest order.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem
from oracle import hp as hpo
from oracle.quadrature import gll, lagrange


def _orders(nx, ny, nz, choices, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(choices, size=nx * ny * nz)


def _assemble(h, vertices, qkind, op, coeff="sine"):
    f = hpo.operator(h, vertices, qkind, op, coeff)
    return np.column_stack([f(np.eye(h.n_true)[:, i]) for i in range(h.n_true)])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_uniform_order_is_the_standard_space(p):
    m = synthetic.HexMesh(2, 2, 1, p, seed=3)
    h = hpo.HpSpace(2, 2, 1, np.full(m.n_elem, p))
    assert h.n_true == m.n_ldof
    # every row of P holds a single 1: the element node is a true dof
    assert np.all(np.diff(h.P.indptr) == 1) and np.all(h.P.data == 1.0)
    perm = np.zeros(m.n_ldof, dtype=np.int64)
    perm[m.elem_dofs.reshape(-1)] = h.P.indices          # lattice node -> true dof
    sp_ = fem.Space(p, "gll")
    A = fem.assemble(sp_, m.elem_dofs, fem.qdata_diffusion(sp_, m.vertices, "sine"), fem.DIFFUSION, m.n_ldof).toarray()
    A_hp = _assemble(h, m.vertices, "gll", fem.DIFFUSION)
    np.testing.assert_allclose(A_hp[np.ix_(perm, perm)], A, atol=1e-13)


def _eval_element(p, values, xi):
    """The element polynomial (nodal values [P^3], a fastest) at reference points xi [n, 3]."""
    x, _ = gll(p + 1)
    La = lagrange(x, xi[:, 0])[0]
    Lb = lagrange(x, xi[:, 1])[0]
    Lc = lagrange(x, xi[:, 2])[0]
    V = values.reshape(p + 1, p + 1, p + 1)   # [c, b, a]
    return np.einsum("na,nb,nc,cba->n", La, Lb, Lc, V)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_orders_are_conforming(seed):
    nx, ny, nz = 3, 3, 2
    orders = _orders(nx, ny, nz, [1, 2, 3, 4], seed)
    h = hpo.HpSpace(nx, ny, nz, orders)
    x = np.random.default_rng(10 + seed).standard_normal(h.n_true)
    vals = hpo.element_values(h, x)
    rng = np.random.default_rng(seed)
    checked = 0
    for e in range(nx * ny * nz):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        for d in range(3):
            c = [ex, ey, ez]
            c[d] += 1
            if c[d] >= (nx, ny, nz)[d]:
                continue
            f = c[0] + nx * (c[1] + ny * c[2])
            pts = rng.uniform(-1, 1, size=(7, 3))
            pa, pb = pts.copy(), pts.copy()
            pa[:, d], pb[:, d] = 1.0, -1.0                  # the shared face seen from both elements
            ua = _eval_element(int(orders[e]), vals[e], pa)
            ub = _eval_element(int(orders[f]), vals[f], pb)
            np.testing.assert_allclose(ua, ub, atol=1e-12)
            checked += 1
    assert checked == 2 * 3 * 2 + 3 * 2 * 2 + 3 * 3 * 1
    # a plain (unconstrained) vector of element values would not be continuous
    assert np.abs(vals[0]).max() > 0


def _true_positions(h, vertices):
    """Physical position of every true dof, from an element node whose row of P is that dof alone."""
    pos = np.full((h.n_true, 3), np.nan)
    for e, p in enumerate(h.orders):
        X = fem.node_points(int(p), vertices[e:e + 1])[0]
        r0 = h.row0[e]
        for n in range(X.shape[0]):
            a, b = h.P.indptr[r0 + n], h.P.indptr[r0 + n + 1]
            if b - a == 1 and h.P.data[a] == 1.0:
                pos[h.P.indices[a]] = X[n]
    assert not np.isnan(pos).any()
    return pos


@pytest.mark.parametrize("seed", [0, 3])
def test_polynomials_of_the_lowest_order_are_reproduced(seed):
    nx, ny, nz = 3, 2, 2
    orders = _orders(nx, ny, nz, [2, 3, 4], seed)
    m = synthetic.HexMesh(nx, ny, nz, 1, seed=0, perturb=0.0)
    h = hpo.HpSpace(nx, ny, nz, orders)
    T = _true_positions(h, m.vertices)
    f = lambda X: 1.0 + X[:, 0] ** 2 * X[:, 1] - 3.0 * X[:, 2] ** 2 + X[:, 0] * X[:, 1] * X[:, 2]
    uE = hpo.element_values(h, f(T))
    for e, p in enumerate(orders):
        X = fem.node_points(int(p), m.vertices[e:e + 1])[0]
        np.testing.assert_allclose(uE[e], f(X), atol=1e-12)


def test_linear_patch_test_and_operator_properties():
    nx, ny, nz = 3, 3, 2
    orders = _orders(nx, ny, nz, [1, 2, 3], 5)
    m = synthetic.HexMesh(nx, ny, nz, 1, seed=4)
    h = hpo.HpSpace(nx, ny, nz, orders)
    A = _assemble(h, m.vertices, "gauss", fem.DIFFUSION, None)
    np.testing.assert_allclose(A, A.T, atol=1e-13)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 * ev.max()
    np.testing.assert_allclose(A @ np.ones(h.n_true), 0.0, atol=1e-12)
    T = _true_positions(h, m.vertices)
    u = T @ np.array([0.7, -1.2, 0.4])
    y = A @ u
    inner = ~h.boundary_mask()
    assert np.abs(y[inner]).max() < 1e-12 * np.abs(y).max()
    assert np.abs(y[~inner]).max() > 1e-3
    M = _assemble(h, m.vertices, "gauss", fem.MASS, None)
    assert abs(np.ones(h.n_true) @ M @ np.ones(h.n_true) - 1.0) < 1e-13


def _solve(N, lo, hi):
    orders = np.array([lo if (e % N) < N // 2 else hi for e in range(N ** 3)])
    m = synthetic.cube_mesh(N, 1, seed=0)
    h = hpo.HpSpace(N, N, N, orders)
    A = sps.csr_matrix(_assemble(h, m.vertices, "gll", fem.DIFFUSION, "sine")).tolil()
    mask = h.boundary_mask()
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    # right-hand side: element loads P^T b_E with the same quadrature
    bE = np.zeros(h.P.shape[0])
    for p in np.unique(orders):
        sel = np.nonzero(orders == p)[0]
        s_ = fem.Space(int(p), "gll")
        X, J = fem.trilinear_map(m.vertices[sel], s_.XI)
        fq = s_.W[None, :] * np.abs(np.linalg.det(J)) * fem.manufactured_source(X, "sine")
        be = np.einsum("qn,eq->en", s_.Phi, fq)
        idx = h.row0[sel][:, None] + np.arange(s_.nd)[None, :]
        bE[idx] = be
    b = h.P.T @ bE
    b[mask] = 0.0
    u = spla.spsolve(A.tocsc(), b)
    uE = hpo.element_values(h, u)
    err2 = 0.0
    for e, p in enumerate(orders):
        s_ = fem.Space(int(p), "gauss", int(p) + 3)
        X, J = fem.trilinear_map(m.vertices[e:e + 1], s_.XI)
        uh = s_.Phi @ uE[e]
        err2 += float(np.sum(s_.W * np.abs(np.linalg.det(J[0])) * (uh - fem.exact_solution(X[0])) ** 2))
    return np.sqrt(err2)


def test_mixed_order_convergence():
    # orders 1 | 2 in two halves of the cube: the error decays at least at the rate of order 1 (h^2)
    e = [_solve(N, 1, 2) for N in (2, 4)]
    rate = np.log(e[0] / e[1]) / np.log(2.0)
    assert rate >= 1.7, (e, rate)

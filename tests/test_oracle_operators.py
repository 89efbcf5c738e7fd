"""Pins for the oracle's dense mass/diffusion actions (Section 2: A_L = block-diag(A^e), A^e = D^T G^e D)."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial

import synthetic
from oracle import fem
from oracle.quadrature import gll


def _mesh_and_space(N, p, qkind, Q=None, seed=0, perturb=0.1):
    m = synthetic.cube_mesh(N, p, seed=seed, perturb=perturb)
    return m, fem.Space(p, qkind, Q)


def _exact_1d(p):
    """1D mass and stiffness of the GLL Lagrange basis on [-1,1], integrated exactly with numpy polynomials."""
    nodes, _ = gll(p + 1)
    polys = []
    for j in range(p + 1):
        others = np.delete(nodes, j)
        lj = Polynomial.fromroots(others)
        polys.append(lj / lj(nodes[j]))
    M = np.zeros((p + 1, p + 1))
    K = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1):
            im = (polys[a] * polys[b]).integ()
            ik = (polys[a].deriv() * polys[b].deriv()).integ()
            M[a, b] = im(1) - im(-1)
            K[a, b] = ik(1) - ik(-1)
    return M, K


def test_mass_total_volume_c1():
    # the mass workload: 4^3 perturbed mesh, Q2 on 3 GLL nodes, 4 Gauss points per direction, rho = 1
    m, sp_ = _mesh_and_space(4, 2, "gauss", 4)
    assert m.n_ldof == 729
    qd = fem.qdata_mass(sp_, m.vertices)
    one = np.ones(m.n_ldof)
    assert abs(one @ fem.apply(sp_, m.elem_dofs, qd, one, fem.MASS) - 1.0) < 1e-14


@pytest.mark.parametrize("p,qkind", [(2, "gll"), (3, "gll"), (4, "gauss"), (1, "gauss")])
def test_mass_volume_other_rules(p, qkind):
    m, sp_ = _mesh_and_space(3, p, qkind, seed=2)
    qd = fem.qdata_mass(sp_, m.vertices)
    one = np.ones(m.n_ldof)
    assert abs(one @ fem.apply(sp_, m.elem_dofs, qd, one, fem.MASS) - 1.0) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_affine_element_matrices_are_kronecker_products(p):
    # unperturbed element of size h: M^e = (h/2)^3 M1 (x) M1 (x) M1,
    # K^e = (h/2) [M1 (x) M1 (x) K1 + M1 (x) K1 (x) M1 + K1 (x) M1 (x) M1] with exact 1D matrices
    # (Gauss with p+1 points integrates both exactly); index n = a + P(b + P c) puts c slowest.
    h = 1.0 / 2
    m, sp_ = _mesh_and_space(2, p, "gauss", p + 1, perturb=0.0)
    M1, K1 = _exact_1d(p)
    Me = fem.element_matrices(sp_, fem.qdata_mass(sp_, m.vertices), fem.MASS)
    Ke = fem.element_matrices(sp_, fem.qdata_diffusion(sp_, m.vertices), fem.DIFFUSION)
    kron3 = lambda A, B, C: np.kron(A, np.kron(B, C))
    np.testing.assert_allclose(Me[3], (h / 2) ** 3 * kron3(M1, M1, M1), atol=1e-15)
    Kref = (h / 2) * (kron3(M1, M1, K1) + kron3(M1, K1, M1) + kron3(K1, M1, M1))
    np.testing.assert_allclose(Ke[5], Kref, atol=1e-13)


def test_q1_collocated_is_seven_point_stencil():
    # p = 1, 2-point GLL (trapezoid) quadrature, k = 1, unperturbed: 1D stiffness (x) lumped masses,
    # which assembles to h times the 7-point finite-difference Laplacian at interior nodes:
    # 6h on the diagonal, -h for each of the 6 neighbours, 0 elsewhere.
    N = 4
    h = 1.0 / N
    m, sp_ = _mesh_and_space(N, 1, "gll", perturb=0.0)
    A = fem.assemble(sp_, m.elem_dofs, fem.qdata_diffusion(sp_, m.vertices), fem.DIFFUSION, m.n_ldof).toarray()
    M = N + 1
    for I, J, K in [(1, 1, 1), (2, 3, 1), (3, 2, 2)]:
        i = I + M * (J + M * K)
        row = A[i].copy()
        assert abs(row[i] - 6 * h) < 1e-14
        for d in (1, M, M * M):
            assert abs(row[i + d] + h) < 1e-14 and abs(row[i - d] + h) < 1e-14
            row[i + d] = row[i - d] = 0
        row[i] = 0
        assert np.abs(row).max() < 1e-14


@pytest.mark.parametrize("p,qkind,coef", [(1, "gll", None), (3, "gll", "sine"), (2, "gauss", "sine"), (4, "gll", None),
                                         (2, "gll", None), (1, "gauss", None)])
def test_diffusion_invariants(p, qkind, coef):
    m, sp_ = _mesh_and_space(3, p, qkind, seed=4)
    G = fem.qdata_diffusion(sp_, m.vertices, coef)
    A = lambda v: fem.apply(sp_, m.elem_dofs, G, v, fem.DIFFUSION)
    n = m.n_ldof
    assert np.abs(A(np.ones(n))).max() < 1e-13
    x = synthetic.uniform(n, seed=1)
    y = synthetic.uniform(n, seed=2)
    assert abs(x @ A(y) - y @ A(x)) < 1e-12 * abs(x @ A(y))
    assert x @ A(x) > 0
    # patch test: a linear function lies in the space; with k = 1 its action is a pure boundary flux, so
    # interior rows vanish whenever the quadrature integrates cofactor(J) * grad(phi) exactly
    # (degree p+1 per direction for a trilinear map: GLL with p+1 points needs p >= 2)
    if coef is None and (p >= 2 or qkind == "gauss"):
        sp_n = fem.Space(p, "gll")
        Xn, _ = fem.trilinear_map(m.vertices, sp_n.XI)
        lin = np.zeros(n)
        lin[m.elem_dofs.reshape(-1)] = (Xn @ np.array([1.0, -2.0, 0.5])).reshape(-1)
        r = A(lin)
        assert np.abs(r[m.boundary == 0]).max() < 1e-12


@pytest.mark.parametrize("p,qkind,op", [(1, "gll", fem.DIFFUSION), (2, "gauss", fem.MASS), (3, "gll", fem.DIFFUSION),
                                       (2, "gauss", fem.DIFFUSION), (4, "gll", fem.MASS)])
def test_dense_action_equals_assembled(p, qkind, op):
    # two oracle paths: matrix-free element loop vs assembled sparse matrix, on 1..8 elements
    for dims in [(1, 1, 1), (2, 1, 1), (2, 2, 2)]:
        m = synthetic.HexMesh(*dims, p, seed=3)
        sp_ = fem.Space(p, qkind)
        qd = fem.qdata_mass(sp_, m.vertices) if op == fem.MASS else fem.qdata_diffusion(sp_, m.vertices, "sine")
        A = fem.assemble(sp_, m.elem_dofs, qd, op, m.n_ldof)
        x = synthetic.uniform(m.n_ldof, seed=9)
        np.testing.assert_allclose(fem.apply(sp_, m.elem_dofs, qd, x, op), A @ x, rtol=0,
                                   atol=1e-14 * np.abs(A).max() * m.n_ldof)
        # Jacobi diagonal: from element diagonals vs the assembled diagonal
        np.testing.assert_allclose(fem.jacobi_diagonal(sp_, m.elem_dofs, qd, op, m.n_ldof), A.diagonal(), rtol=1e-13)
        # several columns at once = column by column
        X = np.stack([x, 2 * x - 1, x ** 2], 1)
        Y = fem.apply(sp_, m.elem_dofs, qd, X, op)
        for c in range(3):
            np.testing.assert_allclose(Y[:, c], A @ X[:, c], atol=1e-13 * np.abs(A).max() * m.n_ldof)


def test_masked_operator():
    m, sp_ = _mesh_and_space(2, 2, "gll")
    G = fem.qdata_diffusion(sp_, m.vertices, "sine")
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).toarray()
    Am = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, G, v, fem.DIFFUSION), m.boundary)
    b = m.boundary.astype(bool)
    ref = A.copy()
    ref[b, :] = 0
    ref[:, b] = 0
    ref[b, b] = 1
    x = synthetic.uniform(m.n_ldof, seed=5)
    np.testing.assert_allclose(Am(x), ref @ x, atol=1e-13)
    d = fem.jacobi_diagonal(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof, mask=m.boundary)
    np.testing.assert_allclose(d, np.diag(ref), rtol=1e-13)


def test_coefficient_scales_linearly():
    m, sp_ = _mesh_and_space(2, 3, "gll")
    k = synthetic.lognormal(m.n_elem * sp_.nq, seed=1).reshape(m.n_elem, sp_.nq)
    G1 = fem.qdata_diffusion(sp_, m.vertices)
    Gk = fem.qdata_diffusion(sp_, m.vertices, k)
    np.testing.assert_allclose(Gk, k[..., None, None] * G1)
    # sine coefficient: 1 + 0.5 sin sin sin evaluated at the mapped quadrature points
    X, _ = fem.trilinear_map(m.vertices, sp_.XI)
    e, q = 5, 17
    x, y, z = X[e, q]
    kk = 1 + 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    np.testing.assert_allclose(fem.qdata_diffusion(sp_, m.vertices, "sine")[e, q], kk * G1[e, q], rtol=1e-15)


def test_cost_model_values():
    # Section 2: reads 7(p+1)^3, flops 12(p+1)^4 + 15(p+1)^3 (first term doubled if not collocated)
    assert fem.cost_model(7) == (3584, 56832)
    assert fem.cost_model(7, collocated=False) == (3584, 105984)
    assert fem.cost_model(1) == (56, 312)


@pytest.mark.parametrize("pc,pf", [(1, 2), (1, 7), (3, 7), (2, 4), (4, 8)])
def test_prolongation_reproduces_coarse_functions(pc, pf):
    # a coarse finite-element function evaluated at the fine nodes: on an affine mesh a polynomial of
    # degree <= pc per direction is reproduced exactly (checked at the fine nodes' physical points)
    mc = synthetic.HexMesh(2, 2, 1, pc, perturb=0.0)
    mf = synthetic.HexMesh(2, 2, 1, pf, perturb=0.0)
    spc, spf = fem.Space(pc, "gll"), fem.Space(pf, "gll")
    Xc, _ = fem.trilinear_map(mc.vertices, spc.XI)
    Xf, _ = fem.trilinear_map(mf.vertices, spf.XI)
    f = lambda X: (X[..., 0] ** pc) * (1 + X[..., 1]) - 2 * X[..., 2] ** min(pc, 2) + 0.5
    uc = np.zeros(mc.n_ldof)
    uc[mc.elem_dofs.reshape(-1)] = f(Xc).reshape(-1)
    uf = fem.prolongate(pc, pf, mc.elem_dofs, mf.elem_dofs, uc, mf.n_ldof)
    ref = np.zeros(mf.n_ldof)
    ref[mf.elem_dofs.reshape(-1)] = f(Xf).reshape(-1)
    np.testing.assert_allclose(uf, ref, atol=1e-13)
    # the restriction is the exact transpose of the assembled prolongation
    rf = synthetic.uniform(mf.n_ldof, seed=3)
    rc = fem.restrict(pc, pf, mc.elem_dofs, mf.elem_dofs, rf, mc.n_ldof)
    v = synthetic.uniform(mc.n_ldof, seed=4)
    Pv = fem.prolongate(pc, pf, mc.elem_dofs, mf.elem_dofs, v, mf.n_ldof)
    assert abs(rc @ v - rf @ Pv) <= 1e-12 * abs(rf @ Pv)
    # element matrix rows sum to one (partition of unity of the coarse basis)
    M = fem.prolongation_element(pc, pf)
    np.testing.assert_allclose(M.sum(1), 1.0, atol=1e-13)

"""Pins for the oracle's overlapping Schwarz / fast-diagonalization smoother.

Independent checks: the 1D extended operators of p = 1 have their closed form; on a uniform
Cartesian mesh with collocated GLL quadrature the global operator is exactly a Kronecker sum, so its
restriction to an interior element's nodes must equal the separable local operator (checked for
non-cubic elements, which also pins the direction of each length scaling); the fast-diagonalization
solve inverts that local operator; the additive smoother is symmetric positive definite on the
non-Dirichlet nodes; and as a CG preconditioner it needs fewer iterations than Jacobi.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem
from oracle import schwarz as sw


def test_reference_1d_p1_closed_form():
    A, B = sw.reference_1d(1)
    np.testing.assert_allclose(A, [[1.0, -0.5], [-0.5, 1.0]], atol=1e-15)
    np.testing.assert_allclose(B, np.diag([2.0, 2.0]), atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_local_operator_is_the_restricted_global_operator(p):
    nx, ny, nz = 3, 4, 5
    m = synthetic.HexMesh(nx, ny, nz, p, seed=0, perturb=0.0)
    sp_ = fem.Space(p, "gll")
    A = fem.assemble(sp_, m.elem_dofs, fem.qdata_diffusion(sp_, m.vertices), fem.DIFFUSION, m.n_ldof).toarray()
    e = 1 + nx * (1 + ny * 1)                         # element (1, 1, 1): interior in every direction
    idx = m.elem_dofs[e]
    h = sw.element_lengths(m.vertices[e:e + 1])[0]
    np.testing.assert_allclose(h, [1 / nx, 1 / ny, 1 / nz], atol=1e-15)
    np.testing.assert_allclose(A[np.ix_(idx, idx)], sw.local_operator(p, h, 1.0), atol=1e-12)


@pytest.mark.parametrize("p", [1, 4, 7])
def test_fast_diagonalization_inverts_the_local_operator(p):
    rng = np.random.default_rng(p)
    h = rng.uniform(0.05, 0.3, size=3)
    k = rng.uniform(0.5, 2.0)
    r = rng.standard_normal((p + 1) ** 3)
    z = sw.local_solve(p, h, k, r)
    np.testing.assert_allclose(sw.local_operator(p, h, k) @ z, r, atol=1e-10 * np.abs(r).max())
    S, lam = sw.fdm_1d(p)
    A, B = sw.reference_1d(p)
    np.testing.assert_allclose(S.T @ B @ S, np.eye(p + 1), atol=1e-12)
    np.testing.assert_allclose(S.T @ A @ S, np.diag(lam), atol=1e-11)


def test_smoother_symmetric_positive_definite():
    p = 2
    m = synthetic.HexMesh(2, 2, 2, p, seed=3)
    M = sw.schwarz(p, m.vertices, m.elem_dofs, m.n_ldof, mask=m.boundary)
    Md = np.column_stack([M(np.eye(m.n_ldof)[:, i]) for i in range(m.n_ldof)])
    np.testing.assert_allclose(Md, Md.T, atol=1e-13)
    inner = ~m.boundary.astype(bool)
    ev = np.linalg.eigvalsh(Md[np.ix_(inner, inner)])
    assert ev.min() > 0
    assert np.abs(Md[~inner]).max() == 0.0


def test_schwarz_preconditioned_cg_beats_jacobi():
    p = 4
    m = synthetic.cube_mesh(4, p, seed=1)
    sp_ = fem.Space(p, "gll")
    G = fem.qdata_diffusion(sp_, m.vertices, "sine")
    mask = m.boundary.astype(bool)
    A = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, G, v, fem.DIFFUSION), mask)
    b = fem.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    dj = fem.jacobi_diagonal(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof, mask=mask)
    _, it_j, _, _ = fem.pcg(A, b, 1.0 / dj, tol=1e-8)
    M = sw.schwarz(p, m.vertices, m.elem_dofs, m.n_ldof, mask=mask)
    # preconditioned CG with z = M r (M symmetric positive definite on the free nodes)
    x = np.zeros_like(b)
    r = b.copy()
    z = M(r) + np.where(mask, r, 0.0)
    d = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    it_s = 0
    while np.linalg.norm(r) > 1e-8 * nb and it_s < 500:
        q = A(d)
        a = rz / (d @ q)
        x += a * d
        r -= a * q
        z = M(r) + np.where(mask, r, 0.0)
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
        it_s += 1
    assert np.linalg.norm(r) <= 1e-8 * nb
    assert it_s < 0.7 * it_j, (it_s, it_j)

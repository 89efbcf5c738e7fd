"""Pins for the oracle's curved (isoparametric, degree-p) geometry.

Independent checks: a trilinear map is reproduced exactly (it lies in Q_p); element volumes by
quadrature of det J equal the divergence-theorem surface integral of the interpolated faces; the
warped unit cube keeps volume 1; the linear patch test holds on curved elements when the
quadrature is exact for its integrand; the manufactured solution converges at O(h^{p+1}).
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem
from oracle.quadrature import gauss, gll, lagrange


def _curved(m, amplitude=0.05):
    xyz = synthetic.bubble_warp(fem.global_node_points(m.p, m.vertices, m.elem_dofs, m.n_ldof), amplitude)
    return xyz, fem.Isoparametric(xyz[m.elem_dofs])


@pytest.mark.parametrize("p,qkind", [(1, "gll"), (2, "gauss"), (3, "gll"), (4, "gauss"), (5, "gauss")])
def test_isoparametric_reproduces_trilinear(p, qkind):
    m = synthetic.HexMesh(3, 2, 2, p, seed=21)
    sp_ = fem.Space(p, qkind)
    iso = fem.Isoparametric(fem.node_points(p, m.vertices))
    X0, J0 = fem.trilinear_map(m.vertices, sp_.XI)
    X1, J1 = fem.element_map(sp_, iso)
    np.testing.assert_allclose(X1, X0, atol=1e-14)
    np.testing.assert_allclose(J1, J0, atol=1e-13)
    # the perturbed trilinear Jacobian is not symmetric, so a transposed J would be caught here
    assert np.abs(J0 - np.swapaxes(J0, -1, -2)).max() > 1e-3
    np.testing.assert_allclose(fem.qdata_diffusion(sp_, iso, "sine"), fem.qdata_diffusion(sp_, m.vertices, "sine"),
                               atol=1e-13)


def test_global_node_points_consistent():
    m = synthetic.HexMesh(2, 3, 2, 3, seed=4)
    xyz = fem.global_node_points(3, m.vertices, m.elem_dofs, m.n_ldof)
    np.testing.assert_allclose(xyz[m.elem_dofs], fem.node_points(3, m.vertices), atol=1e-15)
    w = synthetic.bubble_warp(xyz)
    b = m.boundary.astype(bool)
    np.testing.assert_array_equal(w[b], xyz[b])      # boundary nodes do not move
    assert np.abs(w[~b] - xyz[~b]).max() > 1e-2      # interior nodes do


def _face_volume(coords_e, p):
    """V = 1/3 sum_faces int x . (x_u x x_v) du dv over the element's interpolated faces.

    Each face is the 2D Q_p interpolant of its nodes; the integrand has degree <= 3p - 1 per
    variable, integrated exactly by Gauss with ceil(3p/2) + 1 points.
    """
    P = p + 1
    C = coords_e.reshape(P, P, P, 3)  # [c, b, a, xyz]
    nodes, _ = gll(P)
    g, w = gauss((3 * p + 1) // 2 + 1)
    L, dL = lagrange(nodes, g)        # [npts, P]
    # (face nodes as [u, v] grids, outward sign): r faces (u, v) = (s, t), s faces (t, r), t faces (r, s)
    faces = [(C[:, :, 0, :].transpose(1, 0, 2), -1), (C[:, :, -1, :].transpose(1, 0, 2), 1),
             (C[:, 0, :, :], -1), (C[:, -1, :, :], 1),
             (C[0, :, :, :].transpose(1, 0, 2), -1), (C[-1, :, :, :].transpose(1, 0, 2), 1)]
    vol = 0.0
    for F, sgn in faces:  # F[u_node, v_node, xyz]
        x = np.einsum("iu,jv,uvc->ijc", L, L, F)
        xu = np.einsum("iu,jv,uvc->ijc", dL, L, F)
        xv = np.einsum("iu,jv,uvc->ijc", L, dL, F)
        vol += sgn * np.einsum("i,j,ijc,ijc->", w, w, x, np.cross(xu, xv)) / 3.0
    return vol


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_curved_volumes_by_divergence_theorem(p):
    m = synthetic.cube_mesh(2, p, seed=8)
    _, iso = _curved(m, amplitude=0.08)
    sp_ = fem.Space(p, "gauss", (3 * p + 1) // 2 + 1)  # exact for det J (degree <= 3p - 1)
    _, J = fem.element_map(sp_, iso)
    det = np.linalg.det(J)
    assert det.min() > 0
    vol = (sp_.W[None, :] * det).sum(1)
    ref = np.array([_face_volume(iso.coords[e], p) for e in range(m.n_elem)])
    np.testing.assert_allclose(vol, ref, rtol=1e-13)
    assert np.abs(vol - 1.0 / m.n_elem).max() > 1e-3   # the warp really changed the elements
    assert abs(vol.sum() - 1.0) < 1e-13                 # the boundary is fixed: |Omega| = 1


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_curved_mass_total_volume(p):
    # 1^T M 1 = |Omega| = 1: Gauss q = p + 2 integrates det J (degree <= 3p - 1) exactly for p <= 4
    m = synthetic.cube_mesh(2, p, seed=3)
    _, iso = _curved(m)
    sp_ = fem.Space(p, "gauss")
    qd = fem.qdata_mass(sp_, iso)
    one = np.ones(m.n_ldof)
    assert abs(one @ fem.apply(sp_, m.elem_dofs, qd, one, fem.MASS) - 1.0) < 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_curved_linear_patch_test(p):
    # u = c . x is in the isoparametric space; (A u)_i = int grad phi_i . c = 0 at interior nodes when
    # the quadrature is exact for grad_xi phi_i . adj(J) c (degree <= 3p per variable)
    m = synthetic.cube_mesh(2, p, seed=6)
    xyz, iso = _curved(m, amplitude=0.08)
    sp_ = fem.Space(p, "gauss", (3 * p + 1) // 2 + 1)
    G = fem.qdata_diffusion(sp_, iso)
    u = xyz @ np.array([0.3, -1.1, 0.7])
    y = fem.apply(sp_, m.elem_dofs, G, u, fem.DIFFUSION)
    inner = ~m.boundary.astype(bool)
    assert np.abs(y[inner]).max() < 1e-12 * np.abs(y).max()
    assert np.abs(y[~inner]).max() > 1e-3


def _solve_curved(N, p):
    m = synthetic.cube_mesh(N, p, seed=0)
    _, iso = _curved(m)
    sp_ = fem.Space(p, "gll")
    G = fem.qdata_diffusion(sp_, iso, "sine")
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).tolil()
    mask = m.boundary.astype(bool)
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    b = fem.manufactured_rhs(sp_, iso, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    u = spla.spsolve(A.tocsc(), b)
    return fem.l2_error(p, iso, m.elem_dofs, u)


@pytest.mark.parametrize("p,Ns", [(1, (4, 8)), (2, (4, 8))])
def test_curved_convergence_order(p, Ns):
    e = [_solve_curved(N, p) for N in Ns]
    rate = np.log(e[0] / e[1]) / np.log(Ns[1] / Ns[0])
    assert p + 0.7 <= rate <= p + 1.6, (e, rate)

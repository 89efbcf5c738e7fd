"""Pins for the synthetic meshes and the oracle's trilinear geometry."""
import os

import numpy as np
import pytest

import synthetic
from oracle import fem
from oracle.quadrature import gauss

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bp_dof_counts.txt")


def _dof_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        src, conv, p, dims, cnt = [s.strip() for s in line.split("|")]
        rows.append((src, conv, int(p), tuple(int(t) for t in dims.split()), int(cnt)))
    return rows


@pytest.mark.parametrize("src,conv,p,dims,count", _dof_rows())
def test_dof_counts_match_paper_tables(src, conv, p, dims, count):
    m = synthetic.HexMesh(*dims, p, build_map=False)
    got = m.interior_dof_count() if conv == "interior" else m.n_ldof
    assert got == count, src


def test_generator_deterministic_and_portable():
    a = synthetic.uniform(8, seed=3)
    b = synthetic.uniform(8, seed=3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synthetic.uniform(8, seed=4))
    # SplitMix64 reference outputs for state 0 (published test vector of the generator)
    out = synthetic.splitmix64(np.uint64(0), 0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    z = synthetic.standard_normal(200000, seed=1)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_perturbation_bounds():
    N = 5
    m = synthetic.cube_mesh(N, 2, seed=7)
    X = m.vertex_lattice
    g = np.arange(N + 1) / N
    ref = np.stack(np.broadcast_arrays(g[None, None, :], g[:, None, None] * 0 + g[None, :, None], g[:, None, None]), -1)
    d = X - ref
    inner = np.zeros(X.shape[:3], bool)
    inner[1:N, 1:N, 1:N] = True
    assert np.all(d[~inner] == 0)
    assert np.max(np.abs(d)) <= 0.1 / N + 1e-15
    assert np.max(np.abs(d[inner])) > 0.05 / N


@pytest.mark.parametrize("p", [1, 2, 3])
def test_shared_nodes_coincide(p):
    # every copy of a global node, mapped through its element's trilinear map, is the same point
    m = synthetic.HexMesh(3, 2, 2, p, seed=11)
    sp_ = fem.Space(p, "gll")
    X, _ = fem.trilinear_map(m.vertices, sp_.XI)   # collocated: points are the nodes
    pts = np.zeros((m.n_ldof, 3))
    seen = np.zeros(m.n_ldof, bool)
    for e in range(m.n_elem):
        for n, g in enumerate(m.elem_dofs[e]):
            if seen[g]:
                np.testing.assert_allclose(X[e, n], pts[g], atol=1e-14)
            pts[g], seen[g] = X[e, n], True
    assert seen.all()
    # boundary mask = nodes on the faces of the unit cube
    on_b = np.any((np.abs(pts) < 1e-12) | (np.abs(pts - 1) < 1e-12), axis=1)
    assert np.array_equal(on_b, m.boundary.astype(bool))


def test_affine_jacobian():
    m = synthetic.cube_mesh(4, 2, perturb=0.0)
    sp_ = fem.Space(2, "gauss", 4)
    X, J = fem.trilinear_map(m.vertices, sp_.XI)
    np.testing.assert_allclose(J, np.broadcast_to(np.eye(3) * 0.125, J.shape), atol=1e-15)
    # points of element (1,2,3) are its corner plus (xi+1) h/2
    e = 1 + 4 * (2 + 4 * 3)
    np.testing.assert_allclose(X[e], np.array([0.25, 0.5, 0.75]) + (sp_.XI + 1) * 0.125, atol=1e-15)


def _volume_by_surface(V):
    """Volume of a trilinear hex from the divergence theorem, V = 1/3 sum_faces int x . n dS.

    Each face is a bilinear patch through 4 vertices; x . (x_u x x_v) is a polynomial of
    degree <= 3 per variable, integrated exactly by 3x3 Gauss.
    """
    g, w = gauss(3)
    faces = [((0, 2, 4, 6), -1), ((1, 3, 5, 7), 1), ((0, 1, 4, 5), 1), ((2, 3, 6, 7), -1),
             ((0, 1, 2, 3), -1), ((4, 5, 6, 7), 1)]
    vol = 0.0
    for (a, b, c, d), sgn in faces:
        for iu, u in enumerate(g):
            for iv, v in enumerate(g):
                s, t = (1 + u) / 2, (1 + v) / 2
                x = (1 - s) * (1 - t) * V[a] + s * (1 - t) * V[b] + (1 - s) * t * V[c] + s * t * V[d]
                xu = ((1 - t) * (V[b] - V[a]) + t * (V[d] - V[c])) / 2
                xv = ((1 - s) * (V[c] - V[a]) + s * (V[d] - V[b])) / 2
                vol += sgn * w[iu] * w[iv] * x @ np.cross(xu, xv) / 3
    return vol


def test_element_volumes_and_positive_jacobian():
    m = synthetic.cube_mesh(3, 1, seed=5)
    for kind, Q in (("gauss", 2), ("gll", 3), ("gauss", 4)):
        sp_ = fem.Space(2, kind, Q)
        _, J = fem.trilinear_map(m.vertices, sp_.XI)
        det = np.linalg.det(J)
        assert det.min() > 0
        vol = (sp_.W[None, :] * det).sum(1)
        ref = np.array([_volume_by_surface(m.vertices[e]) for e in range(m.n_elem)])
        np.testing.assert_allclose(vol, ref, rtol=1e-13)
        assert abs(vol.sum() - 1.0) < 1e-13

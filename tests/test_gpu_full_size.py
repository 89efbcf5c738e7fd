"""Parity at the full headline size: 64^3 perturbed hexahedra, p = 7, GLL collocated, diffusion with
k = 1 + 0.5 sin sin sin (90,518,849 DOFs), the mesh, vector and launch configuration that bench.py
times (the autotuned kernel variant).  The oracle cannot run the whole action, so it computes sampled
output entries one by one: y_i = sum over the elements e that contain node i of (A^e u^e)_i, each A^e
u^e by dense quadrature.  The samples include element vertices (8 elements), edge and face nodes (4
and 2) and element-interior nodes (1), on and off the boundary of the cube.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, P_ORDER = 64, 7


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


@pytest.fixture(scope="module")
def headline(ceed):
    m = synthetic.cube_mesh(N, P_ORDER, seed=0)
    mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, P_ORDER, torch.from_numpy(m.elem_dofs).cuda(),
                                torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.boundary).cuda())
    x_host = synthetic.uniform(m.n_ldof, seed=1)
    x = torch.from_numpy(x_host).cuda()
    yield m, mesh, x_host, x
    mesh.close()


def _sample_nodes(rng, n_each=40):
    """Lattice indices (ix, iy, iz) of nodes of every sharing class."""
    L = P_ORDER * N + 1
    picks = []
    for _ in range(n_each):   # element vertices: every index a multiple of p
        picks.append(P_ORDER * rng.integers(0, N + 1, size=3))
    for k in range(n_each):   # face nodes (one index a multiple of p) and edge nodes (two)
        v = rng.integers(0, L, size=3)
        for ax in rng.permutation(3)[:1 + k % 2]:
            v[ax] = P_ORDER * rng.integers(0, N + 1)
        picks.append(v)
    for _ in range(n_each):   # anything
        picks.append(rng.integers(0, L, size=3))
    picks += [np.array([0, 0, 0]), np.array([L - 1, L - 1, L - 1]), np.array([P_ORDER, 0, L - 1])]
    return np.array(picks)


def _oracle_entries(m, x_host, nodes):
    """Sampled entries of A x from the elements that contain each node."""
    L = P_ORDER * N + 1
    P = P_ORDER + 1
    contrib = []   # (sample index, element, local node)
    for s, (ix, iy, iz) in enumerate(nodes):
        axes = []
        for i in (ix, iy, iz):
            cand = [i // P_ORDER - 1, i // P_ORDER] if i % P_ORDER == 0 else [i // P_ORDER]
            axes.append([(c, i - P_ORDER * c) for c in cand if 0 <= c < N])
        for ex, a in axes[0]:
            for ey, b in axes[1]:
                for ez, c in axes[2]:
                    contrib.append((s, ex + N * (ey + N * ez), a + P * (b + P * c)))
    els = np.unique([e for _, e, _ in contrib])
    node_id = nodes[:, 0] + L * (nodes[:, 1] + L * nodes[:, 2])
    # the lattice arithmetic above is checked against the mesh's own restriction
    for s, e, loc in contrib:
        assert m.elem_dofs[e, loc] == node_id[s]
    sp_ = fem.Space(P_ORDER, "gll")
    qd = fem.qdata_diffusion(sp_, m.vertices[els], "sine")
    Ye = fem.element_action(sp_, x_host[m.elem_dofs[els]], qd, fem.DIFFUSION)
    row = {e: r for r, e in enumerate(els)}
    ref = np.zeros(len(nodes))
    for s, e, loc in contrib:
        ref[s] += Ye[row[e], loc]
    counts = np.bincount([s for s, _, _ in contrib], minlength=len(nodes))
    return node_id, ref, counts


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (5, 1e-12), (1, 64 * 8 * 2.0 ** -24), (2, 2e-2)])
def test_headline_apply_sampled(ceed, headline, prec, tol):
    m, mesh, x_host, x = headline
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec, qd)
    y = torch.empty_like(x)
    ceed.ceed_autotune_apply(mesh, ceed.CEED_OP_DIFFUSION, qd, prec, x, y)   # the variant bench.py times
    y.fill_(float("nan"))
    ceed.ceed_apply_diffusion(mesh, qd, prec, x, y)
    torch.cuda.synchronize()
    nodes = _sample_nodes(np.random.default_rng(100 + prec))
    node_id, ref, counts = _oracle_entries(m, x_host, nodes)
    assert set(counts.tolist()) >= {1, 2, 4, 8}
    got = y[torch.from_numpy(node_id).cuda()].cpu().numpy()
    assert np.isfinite(got).all()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # global invariant at full size: A 1 = 0 (rows of the derivative matrix sum to zero)
    if prec in (0, 5):
        ones = torch.ones_like(x)
        ceed.ceed_apply_diffusion(mesh, qd, prec, ones, y)
        torch.cuda.synchronize()
        scale = float(np.abs(ref).max()) / float(np.abs(x_host).max())
        assert float(y.abs().max()) <= 1e-11 * scale
    del qd
    torch.cuda.empty_cache()

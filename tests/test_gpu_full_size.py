"""Parity at full size, in the launch configurations bench.py times.

* The headline: 64^3 perturbed hexahedra, p = 7, GLL collocated, diffusion with k = 1 + 0.5 sin sin
  sin (90,518,849 DOFs), the autotuned apply kernel variant, FP64 / double-float / FP32 / BF16
  quadrature data.
* The batched mixed-order apply: p = 3, 5, 7 on 48^3, 40^3, 32^3 (Gauss q = p + 2), 3 components,
  4, 8 and 16 right-hand sides, one autotuned persistent launch.
* The adjoint: p = 4 on 32^3 with a lognormal per-point coefficient, geometry stored and recomputed.

The oracle cannot run whole actions at these sizes, so it computes sampled output entries one by
one: y_i = sum over the elements e that contain node i of (A^e u^e)_i, each A^e u^e by dense
quadrature (and dL/dk on sampled elements, which is elementwise).  The samples include element
vertices (8 elements), edge and face nodes (4 and 2) and element-interior nodes (1), on and off the
boundary of the cube.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _sample_nodes(rng, N, p, n_each=40):
    """Lattice indices (ix, iy, iz) of nodes of every sharing class."""
    L = p * N + 1
    picks = []
    for _ in range(n_each):   # element vertices: every index a multiple of p
        picks.append(p * rng.integers(0, N + 1, size=3))
    for k in range(n_each):   # face nodes (one index a multiple of p) and edge nodes (two)
        v = rng.integers(0, L, size=3)
        for ax in rng.permutation(3)[:1 + k % 2]:
            v[ax] = p * rng.integers(0, N + 1)
        picks.append(v)
    for _ in range(n_each):   # anything
        picks.append(rng.integers(0, L, size=3))
    picks += [np.array([0, 0, 0]), np.array([L - 1, L - 1, L - 1]), np.array([p, 0, L - 1])]
    return np.array(picks)


def _sampled_action(m, N, p, nodes, X, qd_of):
    """Entries (A X)[node] for the sampled lattice nodes; X is [n] or [n, m] (A acts on each column).
    qd_of(els) gives the oracle's diffusion quadrature data of those elements.  Returns (node ids,
    entries, number of elements containing each node)."""
    L, P = p * N + 1, p + 1
    contrib = []   # (sample index, element, local node)
    for s, (ix, iy, iz) in enumerate(nodes):
        axes = []
        for i in (ix, iy, iz):
            cand = [i // p - 1, i // p] if i % p == 0 else [i // p]
            axes.append([(c, i - p * c) for c in cand if 0 <= c < N])
        for ex, a in axes[0]:
            for ey, b in axes[1]:
                for ez, c in axes[2]:
                    contrib.append((s, ex + N * (ey + N * ez), a + P * (b + P * c)))
    els = np.unique([e for _, e, _ in contrib])
    node_id = nodes[:, 0] + L * (nodes[:, 1] + L * nodes[:, 2])
    for s, e, loc in contrib:   # the lattice arithmetic above agrees with the mesh's own restriction
        assert m.elem_dofs[e, loc] == node_id[s]
    Ye = fem.element_action(fem.Space(p, qd_of.qkind), X[m.elem_dofs[els]], qd_of(els), fem.DIFFUSION)
    row = {e: r for r, e in enumerate(els)}
    ref = np.zeros((len(nodes),) + X.shape[1:])
    for s, e, loc in contrib:
        ref[s] += Ye[row[e], loc]
    counts = np.bincount([s for s, _, _ in contrib], minlength=len(nodes))
    return node_id, ref, counts


class _SineQdata:
    def __init__(self, m, p, qkind):
        self.m, self.sp, self.qkind = m, fem.Space(p, qkind), qkind

    def __call__(self, els):
        return fem.qdata_diffusion(self.sp, self.m.vertices[els], "sine")


def _close(got, ref, tol):
    assert np.isfinite(got).all()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.fixture(scope="module")
def headline(ceed):
    N, p = 64, 7
    m = synthetic.cube_mesh(N, p, seed=0)
    mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, p, torch.from_numpy(m.elem_dofs).cuda(),
                                torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.boundary).cuda())
    x_host = synthetic.uniform(m.n_ldof, seed=1)
    x = torch.from_numpy(x_host).cuda()
    yield m, mesh, x_host, x
    mesh.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (5, 1e-12), (1, 64 * 8 * 2.0 ** -24), (2, 2e-2)])
def test_headline_apply_sampled(ceed, headline, prec, tol):
    N, p = 64, 7
    m, mesh, x_host, x = headline
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec, qd)
    y = torch.empty_like(x)
    ceed.ceed_autotune_apply(mesh, ceed.CEED_OP_DIFFUSION, qd, prec, x, y)   # the variant bench.py times
    y.fill_(float("nan"))
    ceed.ceed_apply_diffusion(mesh, qd, prec, x, y)
    torch.cuda.synchronize()
    nodes = _sample_nodes(np.random.default_rng(100 + prec), N, p)
    node_id, ref, counts = _sampled_action(m, N, p, nodes, x_host, _SineQdata(m, p, "gll"))
    assert set(counts.tolist()) >= {1, 2, 4, 8}
    _close(y[torch.from_numpy(node_id).cuda()].cpu().numpy(), ref, tol)
    # global invariant at full size: A 1 = 0 (rows of the derivative matrix sum to zero)
    if prec in (0, 5):
        ones = torch.ones_like(x)
        ceed.ceed_apply_diffusion(mesh, qd, prec, ones, y)
        torch.cuda.synchronize()
        scale = float(np.abs(ref).max()) / float(np.abs(x_host).max())
        assert float(y.abs().max()) <= 1e-11 * scale
    del qd
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def batched_meshes(ceed):
    specs, ncomp = [(3, 48), (5, 40), (7, 32)], 3
    ms, meshes, qds = [], [], []
    for p, N in specs:
        m = synthetic.cube_mesh(N, p, seed=0)
        mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, p, torch.from_numpy(m.elem_dofs).cuda(),
                                    torch.from_numpy(m.vertices).cuda(), None, q_rule=ceed.CEED_QRULE_GAUSS,
                                    ncomp=ncomp)
        qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
        ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
        ms.append(m)
        meshes.append(mesh)
        qds.append(qd)
    yield specs, ncomp, ms, meshes, qds
    for mesh in meshes:
        mesh.close()


@pytest.mark.parametrize("nrhs,prec", [(4, 0), (8, 0), (16, 0), (4, 5)])
def test_batched_mixed_order_sampled(ceed, batched_meshes, nrhs, prec):
    """Every right-hand-side count bench.py times except 1 (covered by the single-mesh tests);
    nrhs = 16 is 48 interleaved columns per node (x and y: 17 GB on the device); prec 5 is the
    double-float FP64-accurate operator in the same persistent launch."""
    specs, ncomp, ms, meshes, qds = batched_meshes
    if prec != 0:
        qds = []
        for mesh in meshes:
            qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec)
            ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec, qd)
            qds.append(qd)
    xs_host, xs, ys = [], [], []
    for k, m in enumerate(ms):
        xh = synthetic.uniform(m.n_ldof * ncomp * nrhs, seed=7 + k)
        xs_host.append(xh)
        xs.append(torch.from_numpy(xh).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
    batch = ceed.ceed_batch_create(meshes, qds, prec, ceed.CEED_OP_DIFFUSION, xs, ys, nrhs=nrhs)
    ceed.ceed_batch_autotune(batch)                      # the launch shape bench.py times
    ceed.ceed_batch_apply(batch)
    ceed.ceed_batch_status(batch)
    for k, ((p, N), m) in enumerate(zip(specs, ms)):
        nodes = _sample_nodes(np.random.default_rng(200 + k + nrhs + prec), N, p, n_each=12)
        X = xs_host[k].reshape(m.n_ldof, ncomp * nrhs)   # [node][component][rhs], A acts on each column
        node_id, ref, counts = _sampled_action(m, N, p, nodes, X, _SineQdata(m, p, "gauss"))
        assert set(counts.tolist()) >= {1, 2, 8}
        got = ys[k].view(m.n_ldof, ncomp * nrhs)[torch.from_numpy(node_id).cuda()].cpu().numpy()
        _close(got, ref, 1e-12)
    batch.close()
    del xs, ys, xs_host
    torch.cuda.empty_cache()


@pytest.mark.parametrize("stored", [True, False])
def test_adjoint_sampled(ceed, stored):
    N, p = 32, 4
    m = synthetic.cube_mesh(N, p, seed=0)
    sp_ = fem.Space(p, "gll")
    mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, p, torch.from_numpy(m.elem_dofs).cuda(),
                                torch.from_numpy(m.vertices).cuda(), None)
    k = synthetic.lognormal(m.n_elem * sp_.nq, seed=3, sigma=0.5).reshape(m.n_elem, sp_.nq)
    x = synthetic.uniform(m.n_ldof, seed=4)
    r = synthetic.uniform(m.n_ldof, seed=5)
    geo = None
    if stored:
        geo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
        ceed.ceed_build_geometry(mesh, geo)
    kd, xd, rd = (torch.from_numpy(a).cuda() for a in (k, x, r))
    dLdx = torch.full_like(xd, float("nan"))
    dLdk = torch.full_like(kd, float("nan"))
    ceed.ceed_apply_diffusion_adjoint(mesh, kd, geo, xd, rd, dLdx, dLdk)
    torch.cuda.synchronize()

    def qd_of(els):
        return k[els][..., None, None] * fem.geometric_factor(sp_, m.vertices[els])
    qd_of.qkind = "gll"
    # dL/dx = A(k) r at sampled nodes
    nodes = _sample_nodes(np.random.default_rng(300), N, p)
    node_id, ref, counts = _sampled_action(m, N, p, nodes, r, qd_of)
    assert set(counts.tolist()) >= {1, 2, 4, 8}
    _close(dLdx[torch.from_numpy(node_id).cuda()].cpu().numpy(), ref, 1e-12)
    # dL/dk on sampled elements (every point): (grad r)^T Ghat (grad x), elementwise
    els = np.sort(np.random.default_rng(301).choice(m.n_elem, size=64, replace=False))
    Gh = fem.geometric_factor(sp_, m.vertices[els])
    gr = np.einsum("dqn,en->edq", sp_.dPhi, r[m.elem_dofs[els]])
    gx = np.einsum("dqn,en->edq", sp_.dPhi, x[m.elem_dofs[els]])
    ref_k = np.einsum("eaq,eqab,ebq->eq", gr, Gh, gx)
    _close(dLdk[torch.from_numpy(els).cuda()].cpu().numpy(), ref_k, 1e-12)
    mesh.close()

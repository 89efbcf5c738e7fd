"""GPU parity of the conforming hp (variable order) operator against the CPU oracle.

The library builds its conforming prolongation P in C++ and the oracle in numpy (oracle.hp), from
the same definition (minimum rule, GLL Lagrange interpolation through lower-order entities) and the
documented true-dof numbering.  Tolerances: P x to 1e-13 (interpolation weights), FP64 operator
1e-12 norm-wise (as for the single-order operator), FP32 element kernels 2e-5.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem
from oracle import hp as hpo
from _util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _group_rows(h):
    """Oracle element-node rows in the library's order (order groups, elements, nodes)."""
    rows = []
    for p in np.unique(h.orders):
        for e in np.nonzero(h.orders == p)[0]:
            rows.append(np.arange(h.row0[e], h.row0[e + 1]))
    return np.concatenate(rows)


def _gpu_hp(ceed, nx, ny, nz, orders, vertices, qkind="gll", dirichlet=True):
    return ceed.ceed_hp_setup(nx, ny, nz, orders, torch.from_numpy(vertices).cuda(),
                              q_rule=ceed.CEED_QRULE_GLL if qkind == "gll" else ceed.CEED_QRULE_GAUSS,
                              dirichlet=dirichlet)


@pytest.mark.parametrize("seed", [0, 1])
def test_prolongation_matches_oracle(ceed, seed):
    nx, ny, nz = 3, 3, 2
    orders = np.random.default_rng(seed).choice([1, 2, 3, 4, 5], size=nx * ny * nz)
    m = synthetic.HexMesh(nx, ny, nz, 1, seed=seed)
    h = hpo.HpSpace(nx, ny, nz, orders)
    g = _gpu_hp(ceed, nx, ny, nz, orders, m.vertices)
    assert g.n_true == h.n_true and g.n_rows == h.P.shape[0] and g.n_groups == len(np.unique(orders))
    x = synthetic.uniform(h.n_true, seed=seed + 3)
    xd = torch.from_numpy(x).cuda()
    ud = torch.empty(g.n_rows, dtype=torch.float64, device="cuda")
    ceed.ceed_hp_prolong(g, xd, ud)
    torch.cuda.synchronize()
    ref = (h.P @ x)[_group_rows(h)]
    np.testing.assert_allclose(ud.cpu().numpy(), ref, atol=1e-13)
    g.close()


CASES = [("diffusion", "gll", True), ("diffusion", "gauss", False), ("mass", "gauss", False), ("mass", "gll", True)]


@pytest.mark.parametrize("prec", ["f64", "f64df"])
@pytest.mark.parametrize("op,qkind,masked", CASES)
def test_apply_matches_oracle(ceed, op, qkind, masked, prec):
    # FP64 and the FP64-accurate double-float element kernels: both within 1e-12 of the oracle
    nx, ny, nz = 3, 2, 2
    orders = np.random.default_rng(7).choice([2, 3, 4, 5, 6], size=nx * ny * nz)
    m = synthetic.HexMesh(nx, ny, nz, 1, seed=2)
    h = hpo.HpSpace(nx, ny, nz, orders)
    g = _gpu_hp(ceed, nx, ny, nz, orders, m.vertices, qkind)
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    cprec = ceed.CEED_F64 if prec == "f64" else ceed.CEED_F64_DF
    ceed.ceed_hp_build_qdata(g, cop, ceed.CEED_COEFF_SINE, prec=cprec)
    x = synthetic.uniform(h.n_true, seed=11)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    ceed.ceed_hp_apply(g, cop, cprec, xd, yd, flags=ceed.CEED_APPLY_DIRICHLET if masked else 0)
    torch.cuda.synchronize()
    f = hpo.operator(h, m.vertices, qkind, fem.DIFFUSION if op == "diffusion" else fem.MASS, "sine")
    ref = fem.masked(f, h.boundary_mask())(x) if masked else f(x)
    assert rel_err(yd.cpu().numpy(), ref) <= 1e-12
    g.close()


def test_orders_357_slabs_and_fp32(ceed):
    # the mixed-order batch workload's orders 3, 5, 7, joined conformingly: x-slabs of a 6x2x2 lattice
    nx, ny, nz = 6, 2, 2
    orders = np.array([3 if (e % nx) < 2 else 5 if (e % nx) < 4 else 7 for e in range(nx * ny * nz)])
    m = synthetic.HexMesh(nx, ny, nz, 1, seed=5)
    h = hpo.HpSpace(nx, ny, nz, orders)
    g = _gpu_hp(ceed, nx, ny, nz, orders, m.vertices, "gauss")
    x = synthetic.uniform(h.n_true, seed=12)
    xd = torch.from_numpy(x).cuda()
    ref = fem.masked(hpo.operator(h, m.vertices, "gauss", fem.DIFFUSION, "sine"), h.boundary_mask())(x)
    for prec, tol in ((ceed.CEED_F64, 1e-12), (ceed.CEED_F64_DF, 1e-12), (ceed.CEED_F32, 2e-5)):
        ceed.ceed_hp_build_qdata(g, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, prec=prec)
        yd = torch.empty_like(xd)
        ceed.ceed_hp_apply(g, ceed.CEED_OP_DIFFUSION, prec, xd, yd, flags=ceed.CEED_APPLY_DIRICHLET)
        torch.cuda.synchronize()
        assert rel_err(yd.cpu().numpy(), ref) <= tol
    g.close()


def test_uniform_order_matches_single_order_mesh(ceed):
    # one order everywhere: the hp operator is the ordinary one (true dofs renumbered)
    p, nx, ny, nz = 4, 3, 2, 2
    m = synthetic.HexMesh(nx, ny, nz, p, seed=9)
    h = hpo.HpSpace(nx, ny, nz, np.full(m.n_elem, p))
    perm = np.zeros(m.n_ldof, dtype=np.int64)
    perm[m.elem_dofs.reshape(-1)] = h.P.indices
    g = _gpu_hp(ceed, nx, ny, nz, np.full(m.n_elem, p), m.vertices, "gll", dirichlet=False)
    ceed.ceed_hp_build_qdata(g, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, prec=ceed.CEED_F64)
    mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, p, torch.from_numpy(m.elem_dofs).cuda(),
                                torch.from_numpy(m.vertices).cuda())
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
    xl = synthetic.uniform(m.n_ldof, seed=4)
    xt = np.empty(h.n_true)
    xt[perm] = xl
    yl = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, torch.from_numpy(xl).cuda(), yl)
    yt = torch.empty(h.n_true, dtype=torch.float64, device="cuda")
    ceed.ceed_hp_apply(g, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64, torch.from_numpy(xt).cuda(), yt)
    torch.cuda.synchronize()
    assert rel_err(yt.cpu().numpy()[perm], yl.cpu().numpy()) <= 1e-13
    g.close()
    mesh.close()

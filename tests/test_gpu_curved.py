"""GPU parity of the curved (isoparametric, degree-p) geometry path against the oracle.

The node positions are built on the host (oracle trilinear nodes moved by the bubble warp) and fed
to both sides, so the two compute the same discrete operator; bar: 1e-12 relative (FP64).
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem
from _util import curved_coords, gpu_mesh, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _qdata(ceed, mesh, op, prec, kind):
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = ceed.alloc_qdata(mesh, cop, prec)
    ceed.ceed_build_qdata(mesh, cop, kind, None, prec, qd)
    return qd


def _apply(ceed, mesh, op, qd, prec, x, flags=0):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    f = ceed.ceed_apply_diffusion if op == "diffusion" else ceed.ceed_apply_mass
    f(mesh, qd, prec, xd, yd, flags=flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


CASES = [(p, q, op) for p in range(1, 9) for q in ("gll", "gauss") for op in ("diffusion", "mass")]


@pytest.mark.parametrize("p,qkind,op", CASES)
def test_curved_apply_matches_oracle(ceed, p, qkind, op):
    dims = (4, 3, 2) if p <= 4 else (3, 2, 2)
    m = synthetic.HexMesh(*dims, p, seed=30 + p)
    xyz = curved_coords(m)
    mesh = gpu_mesh(ceed, m, qkind, coords=xyz)
    sp_ = fem.Space(p, qkind)
    iso = fem.Isoparametric(xyz[m.elem_dofs])
    kind = fem.DIFFUSION if op == "diffusion" else fem.MASS
    if op == "diffusion":
        qref = fem.qdata_diffusion(sp_, iso, "sine")
    else:
        X, _ = fem.element_map(sp_, iso)
        qref = fem.qdata_mass(sp_, iso, fem.coeff_sine(X))
    x = synthetic.uniform(m.n_ldof, seed=40 + p)
    ref = fem.apply(sp_, m.elem_dofs, qref, x, kind)
    qd = _qdata(ceed, mesh, op, ceed.CEED_F64, ceed.CEED_COEFF_SINE)
    y = _apply(ceed, mesh, op, qd, ceed.CEED_F64, x)
    assert rel_err(y, ref) <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # the FP64-accurate double-float operator on the same curved data
    qdf = _qdata(ceed, mesh, op, ceed.CEED_F64_DF, ceed.CEED_COEFF_SINE)
    assert rel_err(_apply(ceed, mesh, op, qdf, ceed.CEED_F64_DF, x), ref) <= 1e-12
    # FP32 operator within its rounding bound
    q32 = _qdata(ceed, mesh, op, ceed.CEED_F32, ceed.CEED_COEFF_SINE)
    assert rel_err(_apply(ceed, mesh, op, q32, ceed.CEED_F32, x), ref) <= 64 * (p + 1) * 2.0 ** -24
    mesh.close()


@pytest.mark.parametrize("p", [1, 3, 8])
def test_node_coords(ceed, p):
    m = synthetic.HexMesh(3, 2, 3, p, seed=5)
    ref = fem.global_node_points(p, m.vertices, m.elem_dofs, m.n_ldof)
    mesh = gpu_mesh(ceed, m, "gll")
    out = torch.empty((m.n_ldof, 3), dtype=torch.float64, device="cuda")
    ceed.ceed_mesh_node_coords(mesh, out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-14
    mesh.close()
    xyz = curved_coords(m)
    mesh = gpu_mesh(ceed, m, "gll", coords=xyz)
    ceed.ceed_mesh_node_coords(mesh, out)
    assert np.array_equal(out.cpu().numpy(), xyz)
    mesh.close()


def test_curved_equals_trilinear_when_undeformed(ceed):
    # nodes of the trilinear map as a "curved" geometry give the trilinear operator (Q1 lies in Q_p)
    p = 4
    m = synthetic.HexMesh(3, 3, 2, p, seed=9)
    flat = gpu_mesh(ceed, m, "gauss")
    xyz = torch.empty((m.n_ldof, 3), dtype=torch.float64, device="cuda")
    ceed.ceed_mesh_node_coords(flat, xyz)
    iso = gpu_mesh(ceed, m, "gauss", coords=xyz.cpu().numpy())
    a = _qdata(ceed, flat, "diffusion", ceed.CEED_F64, ceed.CEED_COEFF_SINE).view(torch.float64)
    b = _qdata(ceed, iso, "diffusion", ceed.CEED_F64, ceed.CEED_COEFF_SINE).view(torch.float64)
    assert (a - b).abs().max().item() <= 1e-13 * a.abs().max().item()
    flat.close()
    iso.close()


@pytest.mark.parametrize("qkind", ["gll", "gauss"])
def test_curved_rhs_diagonal_and_cg(ceed, qkind):
    N, p = 3, 3
    m = synthetic.cube_mesh(N, p, seed=2)
    xyz = curved_coords(m)
    mesh = gpu_mesh(ceed, m, qkind, coords=xyz)
    sp_ = fem.Space(p, qkind)
    iso = fem.Isoparametric(xyz[m.elem_dofs])
    mask = m.boundary.astype(bool)
    G = fem.qdata_diffusion(sp_, iso, "sine")
    bref = fem.manufactured_rhs(sp_, iso, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(mesh, ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    assert rel_err(b.cpu().numpy(), bref) <= 1e-12
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64, ceed.CEED_COEFF_SINE)
    d = torch.empty_like(b)
    ceed.ceed_jacobi_diagonal(mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F64, d, flags=ceed.CEED_APPLY_DIRICHLET)
    dref = fem.jacobi_diagonal(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof, mask=mask)
    assert rel_err(d.cpu().numpy(), dref) <= 1e-12
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).tolil()
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    xref = spla.spsolve(A.tocsc(), bref)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, tol=1e-10,
                                 op=ceed.CEED_OP_DIFFUSION, max_iter=5000)
    assert rep["rel_residual"] <= 1e-10
    assert rel_err(x.cpu().numpy(), xref) <= 1e-8
    mesh.close()


def test_curved_adjoint_stored_geometry_and_refusals(ceed):
    p = 3
    m = synthetic.HexMesh(3, 2, 2, p, seed=12)
    xyz = curved_coords(m)
    mesh = gpu_mesh(ceed, m, "gll", coords=xyz)
    sp_ = fem.Space(p, "gll")
    iso = fem.Isoparametric(xyz[m.elem_dofs])
    k = synthetic.lognormal(m.n_elem * sp_.nq, seed=1).reshape(m.n_elem, sp_.nq)
    x = synthetic.uniform(m.n_ldof, seed=2)
    b = synthetic.uniform(m.n_ldof, seed=3)
    geo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    ceed.ceed_build_geometry(mesh, geo)
    kd = torch.from_numpy(k).cuda().requires_grad_(True)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    L = 0.5 * ((ceed.diffusion_k(xd, kd, mesh, geo) - torch.from_numpy(b).cuda()) ** 2).sum()
    L.backward()
    Lref, gx, gk = fem.adjoint(sp_, iso, m.elem_dofs, k, x, b)
    assert abs(L.item() - Lref) <= 1e-12 * abs(Lref)
    assert rel_err(xd.grad.cpu().numpy(), gx) <= 1e-12
    assert rel_err(kd.grad.cpu().numpy(), gk) <= 1e-12
    # the trilinear-only paths refuse a curved mesh
    with pytest.raises(ceed.CeedError):
        _qdata(ceed, mesh, "diffusion", ceed.CEED_F32_GEO, ceed.CEED_COEFF_SINE)
    y = torch.empty_like(xd.detach())
    with pytest.raises(ceed.CeedError):
        ceed.ceed_apply_diffusion_k(mesh, kd.detach(), None, xd.detach(), y)
    mesh.close()

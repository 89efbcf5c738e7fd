"""GPU parity of the p-multigrid transfers and of p-multigrid-preconditioned CG (Section 1: p-multigrid)."""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem
from _util import gpu_mesh, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _levels(ceed, N, orders, seed=0, lo_prec=None):
    ms, meshes, q64, qlo = [], [], [], []
    for p in orders:
        m = synthetic.cube_mesh(N, p, seed=seed)
        mesh = gpu_mesh(ceed, m, "gll")
        qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
        ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
        ms.append(m)
        meshes.append(mesh)
        q64.append(qd)
        if lo_prec is not None:
            ql = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, lo_prec)
            ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, lo_prec, ql)
            qlo.append(ql)
    return ms, meshes, q64, (qlo if lo_prec is not None else None)


def test_transfers_match_oracle(ceed):
    orders = (7, 3, 1)
    ms, meshes, q64, _ = _levels(ceed, 3, orders, seed=2)
    pmg = ceed.ceed_pmg_create(meshes, q64)
    for lvl in range(2):
        mf, mc = ms[lvl], ms[lvl + 1]
        bf, bc = mf.boundary.astype(bool), mc.boundary.astype(bool)
        uc = synthetic.uniform(mc.n_ldof, seed=10 + lvl)
        ucm = np.where(bc, 0.0, uc)
        uf = torch.empty(mf.n_ldof, dtype=torch.float64, device="cuda")
        ceed.ceed_pmg_prolong(pmg, lvl, torch.from_numpy(uc).cuda(), uf)
        ref = fem.prolongate(mc.p, mf.p, mc.elem_dofs, mf.elem_dofs, ucm, mf.n_ldof)
        ref[bf] = 0.0
        assert rel_err(uf.cpu().numpy(), ref) <= 1e-13
        rf = synthetic.uniform(mf.n_ldof, seed=20 + lvl)
        rc = torch.empty(mc.n_ldof, dtype=torch.float64, device="cuda")
        ceed.ceed_pmg_restrict(pmg, lvl, torch.from_numpy(rf).cuda(), rc)
        refr = fem.restrict(mc.p, mf.p, mc.elem_dofs, mf.elem_dofs, np.where(bf, 0.0, rf), mc.n_ldof)
        refr[bc] = 0.0
        assert rel_err(rc.cpu().numpy(), refr) <= 1e-13
    for k in range(2):
        assert ceed.ceed_pmg_info(pmg, k) > 1.0
    pmg.close()


@pytest.mark.parametrize("lo_prec", [None, 1])
def test_pmg_cg_solves_to_tolerance(ceed, lo_prec):
    N, orders = 4, (5, 2, 1)
    ms, meshes, q64, qlo = _levels(ceed, N, orders, seed=1, lo_prec=lo_prec)
    m = ms[0]
    pmg = ceed.ceed_pmg_create(meshes, q64, qlo, prec_lo=lo_prec or 1)
    b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(meshes[0], ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(meshes[0], q64[0], ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, tol=1e-10,
                                 op=ceed.CEED_OP_DIFFUSION, pmg=pmg)
    assert rep["rel_residual"] <= 1e-10
    st2, rep_j = ceed.ceed_cg_solve(meshes[0], q64[0], ceed.CEED_F64, b, torch.empty_like(b), mode=ceed.CEED_CG_FP64,
                                    tol=1e-10, op=ceed.CEED_OP_DIFFUSION)
    assert rep["iterations"] * 4 < rep_j["iterations"], (rep, rep_j)
    # the same solution as a sparse direct solve of the oracle's assembled system
    sp_ = fem.Space(m.p, "gll")
    G = fem.qdata_diffusion(sp_, m.vertices, "sine")
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).tolil()
    mask = m.boundary.astype(bool)
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    bref = fem.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    xref = spla.spsolve(A.tocsc(), bref)
    assert rel_err(x.cpu().numpy(), xref) <= 1e-8
    pmg.close()


def test_pmg_rejects_mismatched_levels(ceed):
    ms, meshes, q64, _ = _levels(ceed, 2, (3, 1))
    m2 = synthetic.cube_mesh(3, 1)
    other = gpu_mesh(ceed, m2, "gll")
    with pytest.raises(ceed.CeedError):
        ceed.ceed_pmg_create([meshes[0], other], [q64[0], q64[1]])
    with pytest.raises(ceed.CeedError):      # coarse level of higher order
        ceed.ceed_pmg_create([meshes[1], meshes[0]], [q64[1], q64[0]])

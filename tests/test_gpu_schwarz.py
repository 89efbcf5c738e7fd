"""GPU parity of the overlapping Schwarz / fast-diagonalization smoother against the CPU oracle, and
p-multigrid with Chebyshev-Schwarz smoothing.

The library computes the 1D fast-diagonalization basis with its own Jacobi eigensolver (C++) and
applies the smoother in FP32 arithmetic; the oracle uses scipy's generalized eigensolver in FP64.
The smoother is invariant under the choice of eigenvectors, so the two must agree to FP32 rounding
of ~7 passes of (p+1) terms: 1e-5 norm-wise.
"""
import numpy as np
import pytest

import synthetic
from oracle import schwarz as sw
from _util import gpu_mesh, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


@pytest.mark.parametrize("p", [1, 2, 4, 7, 8])
@pytest.mark.parametrize("masked", [False, True])
def test_schwarz_matches_oracle(ceed, p, masked):
    m = synthetic.HexMesh(3, 2, 2, p, seed=p)
    mesh = gpu_mesh(ceed, m, "gll")
    s = ceed.ceed_schwarz_create(mesh, ceed.CEED_COEFF_SINE)
    r = synthetic.uniform(m.n_ldof, seed=30 + p)
    z = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_schwarz_apply(s, torch.from_numpy(r).cuda(), z, flags=ceed.CEED_APPLY_DIRICHLET if masked else 0)
    torch.cuda.synchronize()
    ref = sw.schwarz(p, m.vertices, m.elem_dofs, m.n_ldof, mask=m.boundary if masked else None)(r)
    assert rel_err(z.cpu().numpy(), ref) <= 1e-5
    if masked:
        assert np.abs(z.cpu().numpy()[m.boundary.astype(bool)]).max() == 0.0
    s.close()
    mesh.close()


def test_pmg_with_schwarz_smoothing(ceed):
    N, orders = 4, (5, 2, 1)
    meshes, q64 = [], []
    for p in orders:
        mm = synthetic.cube_mesh(N, p, seed=1)
        mesh = gpu_mesh(ceed, mm, "gll")
        qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
        ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
        meshes.append(mesh)
        q64.append(qd)
    n = meshes[0].n_ldof
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(meshes[0], ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    its = {}
    for smoother in (0, 1):
        pmg = ceed.ceed_pmg_create(meshes, q64, smoother=smoother, smooth_degree=2)
        x = torch.empty_like(b)
        st, rep = ceed.ceed_cg_solve(meshes[0], q64[0], ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, tol=1e-10,
                                     op=ceed.CEED_OP_DIFFUSION, pmg=pmg)
        assert rep["rel_residual"] <= 1e-10
        its[smoother] = rep["iterations"]
        lam = ceed.ceed_pmg_info(pmg, 0)
        assert 0.5 < lam < 4.0
        pmg.close()
    # a better smoother: no more iterations than Chebyshev-Jacobi of the same degree
    assert its[1] <= its[0], its

"""GPU parity of the batched persistent apply (several meshes of different order in one launch)."""
import numpy as np
import pytest

import synthetic
from oracle import fem
from _util import gpu_mesh, oracle_qdata, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _case(ceed, specs, qkind, op, prec, ncomp, nrhs):
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    ms, meshes, qds, xs, ys = [], [], [], [], []
    for k, (p, dims) in enumerate(specs):
        m = synthetic.HexMesh(*dims, p, seed=30 + k)
        mesh = gpu_mesh(ceed, m, qkind, ncomp=ncomp)
        qd = ceed.alloc_qdata(mesh, cop, prec)
        ceed.ceed_build_qdata(mesh, cop, ceed.CEED_COEFF_SINE, None, prec, qd)
        x = torch.from_numpy(synthetic.uniform(m.n_ldof * ncomp * nrhs, seed=40 + k)).cuda()
        ms.append(m)
        meshes.append(mesh)
        qds.append(qd)
        xs.append(x)
        ys.append(torch.full_like(x, np.nan))
    return cop, ms, meshes, qds, xs, ys


@pytest.mark.parametrize("specs,qkind,op,prec,ncomp,nrhs", [
    ([(3, (4, 3, 3)), (5, (3, 2, 2)), (7, (2, 2, 2))], "gauss", "diffusion", 0, 3, 2),
    # the right-hand-side counts bench.py times: 3 components x 8 and x 16 (48 interleaved columns)
    ([(3, (4, 3, 3)), (5, (3, 2, 2)), (7, (2, 2, 2))], "gauss", "diffusion", 0, 3, 8),
    ([(3, (4, 3, 3)), (5, (3, 2, 2)), (7, (2, 2, 2))], "gauss", "diffusion", 0, 3, 16),
    ([(3, (4, 3, 3)), (7, (2, 2, 2))], "gauss", "diffusion", 1, 3, 16),
    # the FP64-accurate double-float operator in the persistent launch
    ([(3, (4, 3, 3)), (5, (3, 2, 2)), (7, (2, 2, 2))], "gauss", "diffusion", 5, 3, 4),
    ([(2, (3, 3, 2)), (8, (2, 2, 1))], "gll", "diffusion", 5, 1, 2),
    ([(3, (3, 3, 3)), (5, (2, 2, 3))], "gauss", "mass", 5, 3, 1),
    ([(2, (3, 3, 2)), (4, (2, 3, 2))], "gll", "diffusion", 0, 1, 4),
    ([(3, (3, 3, 3)), (5, (2, 2, 3))], "gauss", "mass", 0, 3, 1),
    ([(3, (4, 3, 3)), (7, (2, 2, 2))], "gauss", "diffusion", 1, 3, 1),
])
def test_batch_matches_single_mesh_and_oracle(ceed, specs, qkind, op, prec, ncomp, nrhs):
    cop, ms, meshes, qds, xs, ys = _case(ceed, specs, qkind, op, prec, ncomp, nrhs)
    f = ceed.ceed_apply_diffusion if op == "diffusion" else ceed.ceed_apply_mass
    singles = []
    for mesh, qd, x in zip(meshes, qds, xs):
        y = torch.empty_like(x)
        f(mesh, qd, prec, x, y, nrhs=nrhs)
        singles.append(y)
    batch = ceed.ceed_batch_create(meshes, qds, prec, cop, xs, ys, nrhs=nrhs)
    threads, stage, grid = ceed.ceed_batch_info(batch)
    assert grid >= 152 and threads in (128, 192, 256)
    for rep in range(2):
        ceed.ceed_batch_apply(batch)
        ceed.ceed_batch_status(batch)
        for y, ys1 in zip(ys, singles):
            assert torch.equal(y, ys1), "batched and single-mesh applies differ"
    ms_best = ceed.ceed_batch_autotune(batch)
    assert ms_best > 0
    for y in ys:
        y.fill_(np.nan)
    ceed.ceed_batch_apply(batch)
    ceed.ceed_batch_status(batch)
    for y, ys1 in zip(ys, singles):
        assert torch.equal(y, ys1)
    if prec in (0, 5):
        ncol = ncomp * nrhs
        for m, x, y in zip(ms, xs, ys):
            sp_, qref = oracle_qdata(m, qkind, op, "sine")
            X = x.cpu().numpy().reshape(m.n_ldof, ncol)
            ref = fem.apply(sp_, m.elem_dofs, qref, X, fem.DIFFUSION if op == "diffusion" else fem.MASS)
            assert rel_err(y.cpu().numpy().reshape(m.n_ldof, ncol), ref) <= 1e-12
    batch.close()
    for mesh in meshes:
        mesh.close()


def test_batch_rejects_bad_input(ceed):
    cop, ms, meshes, qds, xs, ys = _case(ceed, [(2, (2, 2, 2))], "gll", "diffusion", 0, 1, 1)
    _, _, meshes2, qds2, xs2, ys2 = _case(ceed, [(2, (2, 2, 2))], "gauss", "diffusion", 0, 1, 1)
    with pytest.raises(ceed.CeedError):      # mixed quadrature rules
        ceed.ceed_batch_create(meshes + meshes2, qds + qds2, 0, cop, xs + xs2, ys + ys2)
    with pytest.raises(ceed.CeedError):      # x aliases y
        ceed.ceed_batch_create(meshes, qds, 0, cop, xs, xs)
    with pytest.raises(ceed.CeedError):      # BF16 batches are not supported
        ceed.ceed_batch_create(meshes, qds, 2, cop, xs, ys)

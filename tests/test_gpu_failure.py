"""Failure paths on the GPU, driven in forms that fault, trap and hang nothing.

* Bounded device waits: a test sets the wait limits to 0 polls (ceed_set_wait_limits), so the apply
  kernel's wait for its quadrature-data copy and the persistent batched launch's grid barrier give
  up at once.  The kernels then record CEED_ERR_TIMEOUT and finish (an element whose wait gave up
  writes nothing and waits, with the default bound, for its copy before the block exits); the next
  status call reports it, and after the limits are restored the same mesh or a new batch computes
  the oracle's result again.
* Non-finite input: a NaN or Inf made on the host in b or in the initial guess makes ceed_cg_solve
  return CEED_ERR_NONFINITE in every mode; a clean solve afterwards converges.
"""
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
    yield c
    c.ceed_set_wait_limits(-1, -1)


def _diffusion_case(ceed, dims, p, qkind, seed, ncomp=1, nrhs=1):
    m = synthetic.HexMesh(*dims, p, seed=seed)
    mesh = gpu_mesh(ceed, m, qkind, ncomp=ncomp)
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof * ncomp * nrhs, seed=seed + 1)).cuda()
    return m, mesh, qd, x


@pytest.mark.parametrize("prec", [0, 1, 5])
def test_copy_wait_expiry_then_recovery(ceed, prec):
    m, mesh, _, x = _diffusion_case(ceed, (4, 3, 3), 3, "gll", seed=61)
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec, qd)
    ceed.ceed_set_apply_variant(mesh, ceed.CEED_OP_DIFFUSION, prec, 2, 1)   # TMA-staged variant: it waits
    y = torch.zeros_like(x)
    ceed.ceed_set_wait_limits(0, -1)
    try:
        ceed.ceed_apply_diffusion(mesh, qd, prec, x, y)
        with pytest.raises(ceed.CeedError) as ei:
            ceed.ceed_mesh_status(mesh)
        assert ei.value.status == ceed.CEED_ERR_TIMEOUT
    finally:
        ceed.ceed_set_wait_limits(-1, -1)
    ceed.ceed_mesh_status(mesh)          # the flag was cleared by the report
    y.fill_(float("nan"))
    ceed.ceed_apply_diffusion(mesh, qd, prec, x, y)
    ceed.ceed_mesh_status(mesh)
    sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
    ref = fem.apply(sp_, m.elem_dofs, qref, x.cpu().numpy(), fem.DIFFUSION)
    tol = 1e-12 if prec in (0, 5) else 64 * 4 * 2.0 ** -24
    assert rel_err(y.cpu().numpy(), ref) <= tol
    mesh.close()


@pytest.mark.parametrize("limits", [(-1, 0), (0, -1)])
def test_batch_wait_expiry_then_recovery(ceed, limits):
    """(-1, 0): the grid barrier between colours gives up; (0, -1): the staged copy waits give up."""
    cases = [_diffusion_case(ceed, (4, 3, 3), 3, "gauss", seed=71), _diffusion_case(ceed, (2, 2, 3), 5, "gauss", seed=73)]
    meshes = [c[1] for c in cases]
    qds = [c[2] for c in cases]
    xs = [c[3] for c in cases]
    singles = []
    for mesh, qd, x in zip(meshes, qds, xs):
        y = torch.empty_like(x)
        ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, x, y)
        singles.append(y)
    ys = [torch.zeros_like(x) for x in xs]
    ceed.ceed_set_wait_limits(*limits)
    try:
        batch = ceed.ceed_batch_create(meshes, qds, ceed.CEED_F64, ceed.CEED_OP_DIFFUSION, xs, ys)  # graph keeps these limits
        _, stage, _ = ceed.ceed_batch_info(batch)
        assert stage == 1
        ceed.ceed_batch_apply(batch)
        with pytest.raises(ceed.CeedError) as ei:
            ceed.ceed_batch_status(batch)
        assert ei.value.status == ceed.CEED_ERR_TIMEOUT
        batch.close()
    finally:
        ceed.ceed_set_wait_limits(-1, -1)
    for y in ys:
        y.fill_(float("nan"))
    batch = ceed.ceed_batch_create(meshes, qds, ceed.CEED_F64, ceed.CEED_OP_DIFFUSION, xs, ys)
    for _ in range(2):
        ceed.ceed_batch_apply(batch)
        ceed.ceed_batch_status(batch)
        for y, y1 in zip(ys, singles):
            assert torch.equal(y, y1)
    batch.close()
    for mesh in meshes:
        mesh.close()


def _cg_setup(ceed, N=3, p=3):
    m = synthetic.cube_mesh(N, p, seed=0)
    mesh = gpu_mesh(ceed, m, "gll")
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
    q32 = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F32, q32)
    b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(mesh, ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    return m, mesh, qd, q32, b


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("where,bad", [("b", float("nan")), ("b", float("inf")), ("x0", float("nan"))])
def test_cg_nonfinite_input(ceed, mode, where, bad):
    m, mesh, qd, q32, b = _cg_setup(ceed)
    kw = dict(mode=mode, tol=1e-10, max_iter=2000, op=ceed.CEED_OP_DIFFUSION, raise_on_error=False)
    if mode != ceed.CEED_CG_FP64:
        kw.update(qdata_lo=q32, prec_lo=ceed.CEED_F32)
    interior = int(np.flatnonzero(m.boundary == 0)[len(np.flatnonzero(m.boundary == 0)) // 2])
    bb = b.clone()
    x = torch.zeros_like(b)
    if where == "b":
        bb[interior] = bad                    # made on the host side of the call, before the solve
    else:
        x[interior] = bad
        kw["use_x0"] = 1
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, bb, x, **kw)
    assert st == ceed.CEED_ERR_NONFINITE
    # a clean solve on the same mesh and workspace sizes converges afterwards
    kw.pop("use_x0", None)
    x.zero_()
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, **kw)
    assert st == ceed.CEED_OK and rep["rel_residual"] <= 1e-10
    mesh.close()


def test_fma_throughput_is_plausible(ceed):
    """The measured FMA rates that bench.py divides by: FP64 far below FP32 on GB300, clock in range."""
    f64, f64_clk, mhz64 = ceed.ceed_fma_throughput(0)
    f32, f32_clk, mhz32 = ceed.ceed_fma_throughput(1)
    f32x2, f32x2_clk, _ = ceed.ceed_fma_throughput(2)
    assert 0.05 < f64 < 20 and 5 < f32 < 400 and 5 < f32x2 < 800
    assert f32 > 10 * f64
    assert 300 < mhz64 < 3500 and 300 < mhz32 < 3500
    assert 0.5 < f32_clk <= 130 and 0.1 < f64_clk < 70
    # the double-float operator's compensated sums: FP32 lane operations, at most the FMA pipe's rate
    d16, d16_clk, _ = ceed.ceed_fma_throughput(3)
    d64, d64_clk, _ = ceed.ceed_fma_throughput(4)
    assert 1 < d16 <= 1.05 * 2 * f32x2 and 1 < d64 <= 1.05 * 2 * f32x2
    assert 1 < d16_clk <= 1.05 * 2 * f32x2_clk and d16_clk <= 1.05 * d64_clk

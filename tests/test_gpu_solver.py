"""GPU parity of the PCG driver, mixed-precision refinement and the adjoint against the CPU oracle."""
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


def _setup(ceed, N, p, seed=0):
    m = synthetic.cube_mesh(N, p, seed=seed)
    mesh = gpu_mesh(ceed, m, "gll")
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F64, qd)
    b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(mesh, ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    return m, mesh, qd, b


def _oracle_solution(m, p):
    sp_ = fem.Space(p, "gll")
    G = fem.qdata_diffusion(sp_, m.vertices, "sine")
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof).tolil()
    mask = m.boundary.astype(bool)
    A[mask, :] = 0
    A[:, mask] = 0
    A = A.tocsr() + sps.diags(mask.astype(float))
    b = fem.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, "sine", mask=mask)
    return A, b, spla.spsolve(A.tocsc(), b)


@pytest.mark.parametrize("N,p", [(3, 3), (4, 2), (2, 7)])
def test_cg_fp64_matches_direct_solve(ceed, N, p):
    m, mesh, qd, b = _setup(ceed, N, p)
    A, bref, xref = _oracle_solution(m, p)
    assert rel_err(b.cpu().numpy(), bref) <= 1e-12
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, tol=1e-10,
                                 op=ceed.CEED_OP_DIFFUSION, max_iter=5000)
    assert rep["rel_residual"] <= 1e-10
    xh = x.cpu().numpy()
    assert np.linalg.norm(bref - A @ xh) <= 1.5e-10 * np.linalg.norm(bref)
    assert rel_err(xh, xref) <= 1e-8
    # the oracle's own PCG on the same system takes a comparable number of iterations
    d = fem.jacobi_diagonal(fem.Space(p, "gll"), m.elem_dofs, fem.qdata_diffusion(fem.Space(p, "gll"), m.vertices, "sine"),
                            fem.DIFFUSION, m.n_ldof, mask=m.boundary)
    # the library's FP64 pass aims at half the tolerance (residual-replacement restarts absorb drift)
    _, it_ref, _, _ = fem.pcg(lambda v: A @ v, bref, 1.0 / d, tol=5e-11, maxit=5000)
    assert abs(rep["iterations"] - it_ref) <= max(3, 0.05 * it_ref)
    assert rep["outer_iterations"] == 1
    mesh.close()


@pytest.mark.parametrize("prec_lo", [1, 2, 3, 4, 5])
def test_mixed_refinement_reaches_fp64_tolerance(ceed, prec_lo):
    N, p = 3, 5
    m, mesh, qd, b = _setup(ceed, N, p)
    A, bref, xref = _oracle_solution(m, p)
    qlo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec_lo)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec_lo, qlo)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED, tol=1e-10,
                                 op=ceed.CEED_OP_DIFFUSION, qdata_lo=qlo, prec_lo=prec_lo, inner_tol=1e-3)
    assert rep["rel_residual"] <= 1e-10 and rep["outer_iterations"] >= 2
    xh = x.cpu().numpy()
    assert np.linalg.norm(bref - A @ xh) <= 1.5e-10 * np.linalg.norm(bref)
    print(f"mixed prec {prec_lo}: outer {rep['outer_iterations']} inner {rep['iterations']}")
    mesh.close()


@pytest.mark.parametrize("prec_lo", [1, 2, 4, 5])
def test_mixed_reliable_reaches_fp64_tolerance(ceed, prec_lo):
    # reliable updates: one PCG run with the low-precision operator, true FP64 residual put in place
    # at every 10x decrease; it reaches the FP64 tolerance in about the FP64 iteration count and in no
    # more iterations than restarted refinement with the same inner operator
    N, p = 3, 5
    m, mesh, qd, b = _setup(ceed, N, p)
    A, bref, xref = _oracle_solution(m, p)
    qlo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec_lo)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec_lo, qlo)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE, tol=1e-10,
                                 op=ceed.CEED_OP_DIFFUSION, qdata_lo=qlo, prec_lo=prec_lo, max_iter=5000)
    assert st == ceed.CEED_OK and rep["rel_residual"] <= 1e-10
    xh = x.cpu().numpy()
    assert np.linalg.norm(bref - A @ xh) <= 1.5e-10 * np.linalg.norm(bref)
    assert rel_err(xh, xref) <= 1e-8
    assert rep["outer_iterations"] >= 2
    _, rep64 = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, torch.empty_like(b), mode=ceed.CEED_CG_FP64,
                                  tol=1e-10, op=ceed.CEED_OP_DIFFUSION)
    _, repm = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, torch.empty_like(b), mode=ceed.CEED_CG_MIXED,
                                 tol=1e-10, op=ceed.CEED_OP_DIFFUSION, qdata_lo=qlo, prec_lo=prec_lo)
    # host checks every 10 iterations: up to 9 iterations past each trigger
    assert rep["iterations"] <= 1.3 * rep64["iterations"] + 10, (rep, rep64)
    assert rep["iterations"] <= repm["iterations"] + 10, (rep, repm)
    print(f"prec {prec_lo}: reliable {rep['iterations']} ({rep['outer_iterations']} true residuals), "
          f"refinement {repm['iterations']}, fp64 {rep64['iterations']}")
    mesh.close()


def test_mixed_modes_reject_bad_options(ceed):
    N, p = 2, 3
    m, mesh, qd, b = _setup(ceed, N, p)
    x = torch.empty_like(b)
    with pytest.raises(ceed.CeedError):          # no low-precision operator
        ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE)
    qlo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F32, qlo)
    for delta in (-0.5, 1.0, 2.0):
        with pytest.raises(ceed.CeedError):
            ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE, qdata_lo=qlo,
                               prec_lo=ceed.CEED_F32, reliable_delta=delta)
    with pytest.raises(ceed.CeedError):
        ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=7)
    mesh.close()
    # an iteration cap reports NOT_CONVERGED with the true residual of the final x filled in (this
    # problem needs about 110 iterations)
    m, mesh, qd, b = _setup(ceed, 3, 5)
    qlo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F32, qlo)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE, qdata_lo=qlo,
                                 prec_lo=ceed.CEED_F32, max_iter=10, op=ceed.CEED_OP_DIFFUSION, raise_on_error=False)
    assert st == ceed.CEED_ERR_NOT_CONVERGED and rep["iterations"] == 10
    A, bref, _ = _oracle_solution(m, 5)
    true_rel = np.linalg.norm(bref - A @ x.cpu().numpy()) / np.linalg.norm(bref)
    assert 0 < rep["rel_residual"] < 1 and abs(rep["rel_residual"] - true_rel) <= 1e-6 * true_rel
    mesh.close()


def test_mixed_reliable_on_an_exactly_converging_problem(ceed):
    # a small symmetric problem whose Krylov space closes within a few iterations: the recurrence
    # residual reaches zero, the device stops and the host certifies with the true residual
    m, mesh, qd, b = _setup(ceed, 2, 3)
    qlo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, ceed.CEED_F32, qlo)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE, qdata_lo=qlo,
                                 prec_lo=ceed.CEED_F32, tol=1e-10, op=ceed.CEED_OP_DIFFUSION)
    A, bref, _ = _oracle_solution(m, 3)
    assert np.linalg.norm(bref - A @ x.cpu().numpy()) <= 1.5e-10 * np.linalg.norm(bref)
    assert st == ceed.CEED_OK and rep["rel_residual"] <= 1e-10
    mesh.close()

def test_cg_fixed_iterations_and_cap(ceed):
    m, mesh, qd, b = _setup(ceed, 3, 4)
    x = torch.empty_like(b)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, fixed_iters=7,
                                 op=ceed.CEED_OP_DIFFUSION)
    assert rep["iterations"] == 7
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_FP64, tol=1e-14, max_iter=5,
                                 op=ceed.CEED_OP_DIFFUSION, raise_on_error=False)
    assert st == ceed.CEED_ERR_NOT_CONVERGED and rep["iterations"] == 5
    mesh.close()


def test_dot_deterministic(ceed):
    n = 1_000_003
    x = torch.from_numpy(synthetic.uniform(n, seed=1)).cuda()
    y = torch.from_numpy(synthetic.uniform(n, seed=2)).cuda()
    work = torch.empty(ceed.ceed_dot_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    vals = []
    for _ in range(3):
        ceed.ceed_dot(x, y, out, work)
        vals.append(out.item())
    assert vals[0] == vals[1] == vals[2]
    ref = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
    assert abs(vals[0] - ref) <= 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("p,stored,df", [(4, True, False), (4, False, False), (8, True, False), (2, False, False),
                                         (4, True, True), (8, True, True), (1, True, True), (6, True, True)])
def test_adjoint_matches_oracle(ceed, p, stored, df):
    # df: the forward operator and the adjoint in FP64-accurate double-float arithmetic (stored
    # geometry), held to the same 1e-12 bounds
    m = synthetic.HexMesh(3, 2, 2, p, seed=11)
    sp_ = fem.Space(p, "gll")
    mesh = gpu_mesh(ceed, m, "gll")
    k = synthetic.lognormal(m.n_elem * sp_.nq, seed=1, sigma=0.5).reshape(m.n_elem, sp_.nq)
    x = synthetic.uniform(m.n_ldof, seed=2)
    b = synthetic.uniform(m.n_ldof, seed=3)
    geo = None
    if stored:
        geo = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
        ceed.ceed_build_geometry(mesh, geo)
    kd = torch.from_numpy(k).cuda()
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    kd.requires_grad_(True)
    y = ceed.diffusion_k(xd, kd, mesh, geo, df)
    bd = torch.from_numpy(b).cuda()
    L = 0.5 * ((y - bd) ** 2).sum()
    L.backward()
    Lref, gx, gk = fem.adjoint(sp_, m.vertices, m.elem_dofs, k, x, b)
    assert abs(L.item() - Lref) <= 1e-12 * abs(Lref)
    assert rel_err(xd.grad.cpu().numpy(), gx) <= 1e-12
    assert rel_err(kd.grad.cpu().numpy(), gk) <= 1e-12
    # directional central difference in k on the GPU path itself (h = 1e-6 relative)
    v = torch.from_numpy(synthetic.uniform(k.size, seed=4).reshape(k.shape)).cuda()
    h = 1e-6 * kd.detach().abs().max() / v.abs().max()
    with torch.no_grad():
        Lp = 0.5 * ((ceed.diffusion_k(xd.detach(), kd.detach() + h * v, mesh, geo, df) - bd) ** 2).sum()
        Lm = 0.5 * ((ceed.diffusion_k(xd.detach(), kd.detach() - h * v, mesh, geo, df) - bd) ** 2).sum()
    fd = ((Lp - Lm) / (2 * h)).item()
    an = (kd.grad * v).sum().item()
    assert abs(fd - an) <= 1e-6 * abs(an)
    if df:  # the flag needs stored geometry, and the adjoint takes no mask
        with pytest.raises(ceed.CeedError):
            ceed.ceed_apply_diffusion_k(mesh, kd.detach(), None, xd.detach(), torch.empty_like(xd),
                                        flags=ceed.CEED_APPLY_F64_DF)
        with pytest.raises(ceed.CeedError):
            ceed.ceed_apply_diffusion_adjoint(mesh, kd.detach(), geo, xd.detach(), bd, torch.empty_like(xd),
                                              torch.empty_like(kd), flags=ceed.CEED_APPLY_DIRICHLET)
    mesh.close()


@pytest.mark.parametrize("mode,prec_lo", [(0, None), (1, 1), (2, 1), (2, 2), (2, 4), (2, 5)])
def test_fused_iteration_matches_separate_kernels(ceed, mode, prec_lo):
    """The fused persistent PCG iteration (one launch per batch of iterations) against the
    separate-kernel iteration: same stopping rules, so the same iteration counts up to rounding-order
    effects, both at 1e-10 on the true FP64 residual, solutions agreeing to the solve's accuracy."""
    m, mesh, qd, b = _setup(ceed, 4, 4)
    kw = dict(mode=mode, tol=1e-10, max_iter=4000, op=ceed.CEED_OP_DIFFUSION)
    if prec_lo is not None:
        ql = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, prec_lo)
        ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_SINE, None, prec_lo, ql)
        kw.update(qdata_lo=ql, prec_lo=prec_lo)
    xf, xs = torch.empty_like(b), torch.empty_like(b)
    st, rf = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, xf, **kw)
    st, rs = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, xs, separate_kernels=1, **kw)
    assert rf["fused"] == 1 and rs["fused"] == 0
    assert rf["rel_residual"] <= 1e-10 and rs["rel_residual"] <= 1e-10
    assert abs(rf["iterations"] - rs["iterations"]) <= max(2, rs["iterations"] // 50)
    assert rel_err(xf.cpu().numpy(), xs.cpu().numpy()) <= 1e-8
    # reproducible: the fused reductions have a fixed order
    x2 = torch.empty_like(b)
    st, r2 = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x2, **kw)
    assert torch.equal(x2, xf) and r2["iterations"] == rf["iterations"]
    mesh.close()


def test_fused_iteration_fixed_iterations(ceed):
    # exactly 25 iterations, in batches of 10 launches (10, 10, 5), equal to the separate kernels'
    # iterate up to rounding order
    m, mesh, qd, b = _setup(ceed, 3, 5)
    xf, xs = torch.empty_like(b), torch.empty_like(b)
    _, rf = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, xf, mode=0, fixed_iters=25, op=ceed.CEED_OP_DIFFUSION)
    _, rs = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, xs, mode=0, fixed_iters=25, op=ceed.CEED_OP_DIFFUSION,
                               separate_kernels=1)
    assert rf["iterations"] == rs["iterations"] == 25 and rf["fused"] == 1
    assert rel_err(xf.cpu().numpy(), xs.cpu().numpy()) <= 1e-9
    mesh.close()


def test_fused_iteration_barrier_expiry(ceed):
    # grid barriers of the fused iteration give up at once: TIMEOUT, no hang; then a normal solve
    m, mesh, qd, b = _setup(ceed, 3, 3)
    x = torch.empty_like(b)
    ceed.ceed_set_wait_limits(-1, 0)
    try:
        st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=0, tol=1e-10, op=ceed.CEED_OP_DIFFUSION,
                                     raise_on_error=False)
        assert st == ceed.CEED_ERR_TIMEOUT
    finally:
        ceed.ceed_set_wait_limits(-1, -1)
    st, rep = ceed.ceed_cg_solve(mesh, qd, ceed.CEED_F64, b, x, mode=0, tol=1e-10, op=ceed.CEED_OP_DIFFUSION)
    assert st == ceed.CEED_OK and rep["rel_residual"] <= 1e-10 and rep["fused"] == 1
    mesh.close()

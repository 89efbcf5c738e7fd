"""GPU parity of the fused mass/diffusion apply against the CPU oracle (Section 2, A_L = block-diag(A^e)).

Tolerance: FP64 path, norm-wise relative error <= 1e-12 (the target the operator is built to); FP32
arithmetic paths are reported against FP64 and bounded by c * p * eps32 with eps32 = 2^-24
(c = 64 for FP32 storage, BF16/FP16 storage add their own rounding of the quadrature data).
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
    return c


def _apply(ceed, mesh, op, qd, prec, x, nrhs=1, flags=0):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    f = ceed.ceed_apply_diffusion if op == "diffusion" else ceed.ceed_apply_mass
    f(mesh, qd, prec, xd, yd, nrhs=nrhs, flags=flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _qdata(ceed, mesh, op, prec, coeff="sine"):
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = ceed.alloc_qdata(mesh, cop, prec)
    kind = {"sine": ceed.CEED_COEFF_SINE, None: ceed.CEED_COEFF_ONE}[coeff]
    ceed.ceed_build_qdata(mesh, cop, kind, None, prec, qd)
    return qd


CASES = [(p, q, op) for p in range(1, 9) for q in ("gll", "gauss") for op in ("diffusion", "mass")]


@pytest.mark.parametrize("p,qkind,op", CASES)
def test_apply_fp64_matches_oracle(ceed, p, qkind, op):
    # 5x3x2 elements: several thread blocks per colour and ragged tails
    dims = (5, 3, 2) if p <= 4 else (3, 2, 2)
    m = synthetic.HexMesh(*dims, p, seed=p)
    mesh = gpu_mesh(ceed, m, qkind)
    qd = _qdata(ceed, mesh, op, ceed.CEED_F64)
    sp_, qref = oracle_qdata(m, qkind, op, "sine")
    x = synthetic.uniform(m.n_ldof, seed=10 + p)
    y = _apply(ceed, mesh, op, qd, ceed.CEED_F64, x)
    ref = fem.apply(sp_, m.elem_dofs, qref, x, fem.DIFFUSION if op == "diffusion" else fem.MASS)
    assert rel_err(y, ref) <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    mesh.close()


@pytest.mark.parametrize("p,qkind,op,prec,bound", [
    (7, "gll", "diffusion", 1, 64 * 8 * 2 ** -24), (3, "gauss", "mass", 1, 64 * 4 * 2 ** -24),
    (7, "gll", "diffusion", 2, 2e-2), (7, "gll", "diffusion", 3, 2e-3), (4, "gauss", "diffusion", 1, 64 * 5 * 2 ** -24),
    (7, "gll", "diffusion", 4, 64 * 8 * 2 ** -24), (3, "gauss", "diffusion", 4, 64 * 4 * 2 ** -24),
    (1, "gll", "diffusion", 4, 64 * 2 * 2 ** -24), (8, "gauss", "diffusion", 4, 64 * 9 * 2 ** -24)])
def test_apply_lowprec_error_bound(ceed, p, qkind, op, prec, bound):
    m = synthetic.HexMesh(3, 3, 2, p, seed=3)
    mesh = gpu_mesh(ceed, m, qkind)
    qd = _qdata(ceed, mesh, op, prec)
    sp_, qref = oracle_qdata(m, qkind, op, "sine")
    x = synthetic.uniform(m.n_ldof, seed=4)
    y = _apply(ceed, mesh, op, qd, prec, x)
    ref = fem.apply(sp_, m.elem_dofs, qref, x, fem.DIFFUSION if op == "diffusion" else fem.MASS)
    err = rel_err(y, ref)
    print(f"prec {prec} p={p} {qkind} {op}: rel err vs FP64 oracle {err:.3e} (bound {bound:.1e})")
    assert err <= bound
    mesh.close()


@pytest.mark.parametrize("ncomp,nrhs,p,qkind", [(3, 1, 3, "gauss"), (1, 4, 5, "gll"), (3, 4, 2, "gll"), (3, 2, 7, "gauss")])
def test_multicomponent_multirhs(ceed, ncomp, nrhs, p, qkind):
    m = synthetic.HexMesh(3, 2, 2, p, seed=5)
    mesh = gpu_mesh(ceed, m, qkind, ncomp=ncomp)
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64)
    sp_, qref = oracle_qdata(m, qkind, "diffusion", "sine")
    ncol = ncomp * nrhs
    X = synthetic.uniform(m.n_ldof * ncol, seed=6).reshape(m.n_ldof, ncol)
    Y = _apply(ceed, mesh, "diffusion", qd, ceed.CEED_F64, X.reshape(-1), nrhs=nrhs).reshape(m.n_ldof, ncol)
    ref = fem.apply(sp_, m.elem_dofs, qref, X, fem.DIFFUSION)
    assert rel_err(Y, ref) <= 1e-12
    mesh.close()


@pytest.mark.parametrize("p,qkind", [(2, "gll"), (5, "gauss"), (7, "gll")])
def test_dirichlet_masked_apply(ceed, p, qkind):
    m = synthetic.HexMesh(3, 3, 2, p, seed=7)
    mesh = gpu_mesh(ceed, m, qkind)
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64)
    sp_, qref = oracle_qdata(m, qkind, "diffusion", "sine")
    x = synthetic.uniform(m.n_ldof, seed=8)
    y = _apply(ceed, mesh, "diffusion", qd, ceed.CEED_F64, x, flags=ceed.CEED_APPLY_DIRICHLET)
    Am = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, qref, v, fem.DIFFUSION), m.boundary)
    assert rel_err(y, Am(x)) <= 1e-12
    mesh.close()


def test_single_element_and_deterministic(ceed):
    for p in (1, 8):
        m = synthetic.HexMesh(1, 1, 1, p, seed=0)
        mesh = gpu_mesh(ceed, m, "gll")
        assert mesh.n_colors == 1
        qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64)
        sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
        x = synthetic.uniform(m.n_ldof, seed=1)
        y = _apply(ceed, mesh, "diffusion", qd, ceed.CEED_F64, x)
        assert rel_err(y, fem.apply(sp_, m.elem_dofs, qref, x, fem.DIFFUSION)) <= 1e-12
        mesh.close()
    # bitwise-identical output over repeated applies (no atomics)
    m = synthetic.HexMesh(4, 4, 3, 4, seed=2)
    mesh = gpu_mesh(ceed, m, "gll")
    assert mesh.n_colors == 8
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=3)).cuda()
    ys = []
    for _ in range(5):
        y = torch.empty_like(x)
        ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, x, y)
        ys.append(y)
    for y in ys[1:]:
        assert torch.equal(y, ys[0])
    mesh.close()


def test_invalid_inputs_are_rejected(ceed):
    m = synthetic.HexMesh(2, 1, 1, 2, seed=0)
    dofs = torch.from_numpy(m.elem_dofs).cuda()
    vert = torch.from_numpy(m.vertices).cuda()
    with pytest.raises(ceed.CeedError) as e:
        ceed.ceed_setup_mesh(0, m.n_ldof, 2, dofs, vert)
    assert e.value.status == ceed.CEED_ERR_INVALID
    with pytest.raises(ceed.CeedError):
        ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, 9, dofs, vert)
    bad = dofs.clone()
    bad[1, 3] = m.n_ldof
    with pytest.raises(ceed.CeedError):
        ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, 2, bad, vert)
    with pytest.raises(ceed.CeedError):      # a node no element references
        ceed.ceed_setup_mesh(m.n_elem, m.n_ldof + 1, 2, dofs, vert)
    # inverted element -> BAD_GEOMETRY from the qdata build
    vflip = vert.clone()
    vflip[0] = vflip[0][[1, 0, 3, 2, 5, 4, 7, 6]]
    mesh = ceed.ceed_setup_mesh(m.n_elem, m.n_ldof, 2, dofs, vflip)
    qd = ceed.alloc_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    with pytest.raises(ceed.CeedError) as e:
        ceed.ceed_build_qdata(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_COEFF_ONE, None, ceed.CEED_F64, qd)
    assert e.value.status == ceed.CEED_ERR_BAD_GEOMETRY
    x = torch.zeros(m.n_ldof, dtype=torch.float64, device="cuda")
    with pytest.raises(ceed.CeedError):       # x and y alias
        ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, x, x)
    with pytest.raises(ceed.CeedError):       # no Dirichlet mask on this mesh
        ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, x, torch.empty_like(x), flags=ceed.CEED_APPLY_DIRICHLET)
    mesh.close()


def test_setup_diagonal_and_rhs(ceed):
    for p, qkind, op in ((4, "gll", "diffusion"), (3, "gauss", "diffusion"), (2, "gauss", "mass"), (5, "gll", "mass")):
        m = synthetic.HexMesh(3, 2, 2, p, seed=9)
        mesh = gpu_mesh(ceed, m, qkind)
        qd = _qdata(ceed, mesh, op, ceed.CEED_F64)
        sp_, qref = oracle_qdata(m, qkind, op, "sine")
        fop = fem.DIFFUSION if op == "diffusion" else fem.MASS
        cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
        for flags in (0, ceed.CEED_APPLY_DIRICHLET):
            d = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
            ceed.ceed_jacobi_diagonal(mesh, cop, qd, ceed.CEED_F64, d, flags=flags)
            ref = fem.jacobi_diagonal(sp_, m.elem_dofs, qref, fop, m.n_ldof, mask=m.boundary if flags else None)
            assert rel_err(d.cpu().numpy(), ref) <= 1e-12
        b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
        ceed.ceed_manufactured_rhs(mesh, ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
        bref = fem.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, "sine", mask=m.boundary)
        assert rel_err(b.cpu().numpy(), bref) <= 1e-12
        mesh.close()


@pytest.mark.parametrize("p,qkind,op,prec", [(7, "gll", "diffusion", 0), (7, "gll", "diffusion", 1),
                                             (3, "gauss", "mass", 0), (5, "gauss", "diffusion", 2), (2, "gll", "diffusion", 1),
                                             (5, "gll", "diffusion", 1), (3, "gll", "diffusion", 2), (1, "gll", "diffusion", 1),
                                             (7, "gll", "diffusion", 4), (4, "gauss", "diffusion", 4),
                                             (7, "gll", "diffusion", 5), (8, "gauss", "diffusion", 5),
                                             (3, "gauss", "mass", 5), (2, "gll", "diffusion", 5),
                                             (1, "gll", "mass", 5), (5, "gll", "mass", 5), (6, "gauss", "diffusion", 5)])
def test_apply_variants_identical_and_autotune(ceed, p, qkind, op, prec):
    # every (elements per block, staging) variant runs the same arithmetic: bitwise-identical output
    m = synthetic.HexMesh(5, 3, 3, p, seed=13)
    mesh = gpu_mesh(ceed, m, qkind)
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = _qdata(ceed, mesh, op, prec)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=14)).cuda()
    f = ceed.ceed_apply_diffusion if op == "diffusion" else ceed.ceed_apply_mass
    outs = []
    ne_max = min(32, max(1, 256 // mesh.Q ** 2))
    for stage in (0, 1):
        ne = 1
        while ne <= ne_max:
            ceed.ceed_set_apply_variant(mesh, cop, prec, ne, stage)
            y = torch.empty_like(x)
            f(mesh, qd, prec, x, y)
            outs.append(y)
            ne *= 2
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    ne, stage, ms = ceed.ceed_autotune_apply(mesh, cop, qd, prec, x, torch.empty_like(x))
    assert 1 <= ne <= ne_max and stage in (0, 1) and ms > 0
    y = torch.empty_like(x)
    f(mesh, qd, prec, x, y)
    assert torch.equal(y, outs[0])
    with pytest.raises(ceed.CeedError):
        ceed.ceed_set_apply_variant(mesh, cop, prec, ne_max + 1, 1)
    with pytest.raises(ceed.CeedError):
        ceed.ceed_set_apply_variant(mesh, cop, prec, 1, 2)
    if prec in (0, 5):
        sp_, qref = oracle_qdata(m, qkind, op, "sine")
        ref = fem.apply(sp_, m.elem_dofs, qref, x.cpu().numpy(), fem.DIFFUSION if op == "diffusion" else fem.MASS)
        assert rel_err(y.cpu().numpy(), ref) <= 1e-12
    mesh.close()


@pytest.mark.parametrize("p,qkind,op", CASES)
def test_apply_double_float_matches_oracle(ceed, p, qkind, op):
    # FP64-accurate operator on the FP32 pipe (double-float values, compensated contractions):
    # the same 1e-12 bar as the FP64 operator, for both operators and both quadrature rules
    dims = (5, 3, 2) if p <= 4 else (3, 2, 2)
    m = synthetic.HexMesh(*dims, p, seed=50 + p)
    mesh = gpu_mesh(ceed, m, qkind)
    kind = fem.DIFFUSION if op == "diffusion" else fem.MASS
    qd = _qdata(ceed, mesh, op, ceed.CEED_F64_DF)
    sp_, qref = oracle_qdata(m, qkind, op, "sine")
    x = synthetic.uniform(m.n_ldof, seed=60 + p)
    y = _apply(ceed, mesh, op, qd, ceed.CEED_F64_DF, x)
    ref = fem.apply(sp_, m.elem_dofs, qref, x, kind)
    err = rel_err(y, ref)
    print(f"double-float p={p} {qkind} {op}: rel err {err:.2e}")
    assert err <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # masked operator and several columns
    ym = _apply(ceed, mesh, op, qd, ceed.CEED_F64_DF, x, flags=ceed.CEED_APPLY_DIRICHLET)
    Am = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, qref, v, kind), m.boundary)
    assert rel_err(ym, Am(x)) <= 1e-12
    X = synthetic.uniform(m.n_ldof * 3, seed=70 + p).reshape(m.n_ldof, 3)
    Y = _apply(ceed, mesh, op, qd, ceed.CEED_F64_DF, X.reshape(-1), nrhs=3).reshape(m.n_ldof, 3)
    assert rel_err(Y, fem.apply(sp_, m.elem_dofs, qref, X, kind)) <= 1e-12
    mesh.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_apply(ceed, pinned):
    # the host-buffer entry point runs the same kernels as the device form: bitwise-identical output,
    # and the oracle's action within the FP64 parity bound
    m = synthetic.HexMesh(3, 2, 2, 4, seed=4)
    mesh = gpu_mesh(ceed, m, "gll", ncomp=1)
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64)
    nrhs = 2
    xh = torch.from_numpy(synthetic.uniform(m.n_ldof * nrhs, seed=9))
    yh = torch.full_like(xh, float("nan"))
    if pinned:
        xh, yh = xh.pin_memory(), yh.pin_memory()
    xd = torch.empty(m.n_ldof * nrhs, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ceed.ceed_apply_host(mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F64, xh, yh, xd, yd, nrhs=nrhs)
    y_ref = torch.empty_like(xd)
    ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F64, xh.cuda(), y_ref, nrhs=nrhs)
    torch.cuda.synchronize()
    assert torch.equal(yh, y_ref.cpu())
    sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
    X = xh.numpy().reshape(m.n_ldof, nrhs)
    Y = yh.numpy().reshape(m.n_ldof, nrhs)
    for c in range(nrhs):
        assert rel_err(Y[:, c], fem.apply(sp_, m.elem_dofs, qref, np.ascontiguousarray(X[:, c]), fem.DIFFUSION)) <= 1e-12
    with pytest.raises(ValueError):          # device tensor passed as a host buffer
        ceed.ceed_apply_host(mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F64, xd, yh, xd, yd, nrhs=nrhs)
    with pytest.raises(ceed.CeedError):      # aliased device buffers
        ceed.ceed_apply_host(mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F64, xh, yh, xd, xd, nrhs=nrhs)
    mesh.close()



@pytest.mark.parametrize("scale", [1e-20, 1e-10, 1.0, 1e20, 1e30])
def test_double_float_input_range(ceed, scale):
    """The double-float operator carries each value as two FP32 words, so it holds the 1e-12 bar only
    while every word stays in the FP32 normal range: inputs from 1e-20 to 1e30 with the quadrature data
    of these meshes (the header states the range; at 1e-30 the low words of the products reach the
    FP32 subnormals and the bar fails on the GB300).  The operator is linear: A (s x) = s (A x)."""
    p = 5
    m = synthetic.HexMesh(3, 3, 2, p, seed=81)
    mesh = gpu_mesh(ceed, m, "gll")
    qd = _qdata(ceed, mesh, "diffusion", ceed.CEED_F64_DF)
    sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
    x = synthetic.uniform(m.n_ldof, seed=82)
    ref = scale * fem.apply(sp_, m.elem_dofs, qref, x, fem.DIFFUSION)
    y = _apply(ceed, mesh, "diffusion", qd, ceed.CEED_F64_DF, scale * x)
    assert rel_err(y, ref) <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    mesh.close()

"""GPU parity of the non-tensor (tetrahedral) operator against the CPU oracle (Section 3: the
basis-agnostic dense element operator of libCEED's non-tensor bases and the MAGMA backend's GEMM
formulation).

The library builds its own basis tables (ceed_simplex_basis) and the oracle its own (oracle.simplex);
both sides then apply the mass and diffusion operators on the same seeded Kuhn-split mesh.
Tolerances (norm-wise relative): FP64 arithmetic, native or emulated on the tensor cores, 1e-12; FP32
arithmetic (fused FP32, SGEMM, BF16x9 emulation) 2e-5, i.e. a few hundred eps32 for sums of
P + 3 Q products; TF32 inputs (10-bit mantissas, eps = 2^-11) 5e-3.
"""
import numpy as np
import pytest

import synthetic
from oracle import fem
from oracle import simplex as sx
from _util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _setup(ceed, m, q, dirichlet=True):
    interp, grad, qw, qref = ceed.ceed_simplex_basis(m.p, q)
    return ceed.ceed_nt_setup(m.n_elem, m.n_ldof, interp, grad, qw, qref, torch.from_numpy(m.elem_dofs).cuda(),
                              torch.from_numpy(m.vertices).cuda(),
                              torch.from_numpy(m.boundary).cuda() if dirichlet else None)


def _qdata(ceed, nt, op, prec, kind=None, coeff=None):
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = ceed.alloc_nt_qdata(nt, cop, prec)
    kind = ceed.CEED_COEFF_SINE if kind is None else kind
    ceed.ceed_nt_build_qdata(nt, cop, kind, coeff, prec, qd)
    return qd


def _apply(ceed, nt, op, qd, prec, x, flags=0):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    ceed.ceed_nt_apply(nt, cop, qd, prec, xd, yd, flags=flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _oracle(m, q, op, x, k="sine", mask=None):
    sp_ = sx.SimplexSpace(m.p, q)
    if op == "diffusion":
        qd, fop = sx.qdata_diffusion(sp_, m.vertices, k), fem.DIFFUSION
    else:
        rho = None
        if isinstance(k, str):
            X, _ = sx.affine_map(m.vertices, sp_.XI)
            rho = fem.coeff_sine(X)
        elif k is not None:
            rho = k
        qd, fop = sx.qdata_mass(sp_, m.vertices, rho), fem.MASS
    f = lambda v: fem.apply(sp_, m.elem_dofs, qd, v, fop)
    return fem.masked(f, mask)(x) if mask is not None else f(x)


CASES = [(p, op) for p in range(1, 7) for op in ("diffusion", "mass")]


@pytest.mark.parametrize("p,op", CASES)
def test_fused_fp64_matches_oracle(ceed, p, op):
    # 72 elements = two full blocks of 32 and a ragged tail of 8
    m = synthetic.TetMesh(3, 2, 2, p, seed=p) if p <= 4 else synthetic.TetMesh(2, 2, 1, p, seed=p)
    q = p + 1
    nt = _setup(ceed, m, q)
    qd = _qdata(ceed, nt, op, ceed.CEED_F64)
    x = synthetic.uniform(m.n_ldof, seed=20 + p)
    y = _apply(ceed, nt, op, qd, ceed.CEED_F64, x)
    ref = _oracle(m, q, op, x)
    assert rel_err(y, ref) <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    nt.close()


@pytest.mark.parametrize("p,op", CASES)
def test_fused_double_float_matches_oracle(ceed, p, op):
    # FP64 accuracy on the FP32 pipe (double-float values, tables and quadrature data; Dot2 sums):
    # held to the FP64 bound against the oracle, and only the fused algorithm exists for it
    m = synthetic.TetMesh(3, 2, 2, p, seed=p) if p <= 4 else synthetic.TetMesh(2, 2, 1, p, seed=p)
    q = p + 1
    nt = _setup(ceed, m, q)
    qd = _qdata(ceed, nt, op, ceed.CEED_F64_DF)
    x = synthetic.uniform(m.n_ldof, seed=20 + p)
    y = _apply(ceed, nt, op, qd, ceed.CEED_F64_DF, x)
    ref = _oracle(m, q, op, x)
    assert rel_err(y, ref) <= 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    with pytest.raises(ceed.CeedError):
        ceed.ceed_nt_set_algorithm(nt, cop, ceed.CEED_F64_DF, ceed.CEED_NT_GEMM, 0, 0)
    nt.close()


GEMM_CASES = [("f64", 0, 1e-12), ("f64", 1, 1e-12), ("f32", 0, 2e-5), ("f32", 1, 2e-5), ("f32", 2, 5e-3)]


@pytest.mark.parametrize("prec,mode,tol", GEMM_CASES)
@pytest.mark.parametrize("op", ["diffusion", "mass"])
def test_gemm_formulation_matches_oracle(ceed, prec, mode, tol, op):
    p, q = 3, 4
    m = synthetic.TetMesh(4, 3, 3, p, seed=11)        # 216 elements
    nt = _setup(ceed, m, q)
    cprec = ceed.CEED_F64 if prec == "f64" else ceed.CEED_F32
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = _qdata(ceed, nt, op, cprec)
    x = synthetic.uniform(m.n_ldof, seed=5)
    ref = _oracle(m, q, op, x)
    for eta in (0, 64, 50):                             # one GEMM; batches of 64 (+ 24); of 50 (+ 16)
        ceed.ceed_nt_set_algorithm(nt, cop, cprec, ceed.CEED_NT_GEMM, eta, mode)
        y = _apply(ceed, nt, op, qd, cprec, x)
        assert rel_err(y, ref) <= tol, (eta, rel_err(y, ref))
    nt.close()


@pytest.mark.parametrize("op", ["diffusion", "mass"])
def test_fused_fp32_matches_oracle(ceed, op):
    p, q = 4, 5
    m = synthetic.TetMesh(3, 3, 2, p, seed=3)
    nt = _setup(ceed, m, q)
    qd = _qdata(ceed, nt, op, ceed.CEED_F32)
    x = synthetic.uniform(m.n_ldof, seed=6)
    y = _apply(ceed, nt, op, qd, ceed.CEED_F32, x)
    assert rel_err(y, _oracle(m, q, op, x)) <= 2e-5
    nt.close()


@pytest.mark.parametrize("p,op", CASES)
def test_tensor_core_matches_oracle(ceed, p, op):
    # tcgen05 kernel, 3xTF32: 360 elements = two full tiles of 128 and a ragged tile of 104 (p <= 4)
    m = synthetic.TetMesh(5, 4, 3, p, seed=30 + p) if p <= 4 else synthetic.TetMesh(4, 3, 2, p, seed=30 + p)
    q = p + 1
    nt = _setup(ceed, m, q)
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = _qdata(ceed, nt, op, ceed.CEED_F32)
    ceed.ceed_nt_set_algorithm(nt, cop, ceed.CEED_F32, ceed.CEED_NT_TC)
    x = synthetic.uniform(m.n_ldof, seed=40 + p)
    ref = _oracle(m, q, op, x)
    for flags in (0, ceed.CEED_APPLY_DIRICHLET):
        y = _apply(ceed, nt, op, qd, ceed.CEED_F32, x, flags=flags)
        ceed.ceed_nt_status(nt)
        r = ref if flags == 0 else _oracle(m, q, op, x, mask=m.boundary)
        assert rel_err(y, r) <= 2e-5, (flags, rel_err(y, r))
    # the same arithmetic on the CUDA cores agrees to FP32 rounding
    ceed.ceed_nt_set_algorithm(nt, cop, ceed.CEED_F32, ceed.CEED_NT_FUSED)
    y2 = _apply(ceed, nt, op, qd, ceed.CEED_F32, x)
    ceed.ceed_nt_set_algorithm(nt, cop, ceed.CEED_F32, ceed.CEED_NT_TC)
    y1 = _apply(ceed, nt, op, qd, ceed.CEED_F32, x)
    assert rel_err(y1, y2) <= 2e-5
    nt.close()


@pytest.mark.parametrize("algo", ["fused", "gemm"])
def test_dirichlet_masked_and_per_point_coefficient(ceed, algo):
    p, q = 2, 3
    m = synthetic.TetMesh(3, 3, 3, p, seed=7)
    nt = _setup(ceed, m, q)
    k = synthetic.lognormal(m.n_elem * q ** 3, seed=9)
    kd = torch.from_numpy(k).cuda()
    qd = _qdata(ceed, nt, "diffusion", ceed.CEED_F64, ceed.CEED_COEFF_PER_QPT, kd)
    if algo == "gemm":
        ceed.ceed_nt_set_algorithm(nt, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64, ceed.CEED_NT_GEMM, 0, 0)
    x = synthetic.uniform(m.n_ldof, seed=8)
    y = _apply(ceed, nt, "diffusion", qd, ceed.CEED_F64, x, flags=ceed.CEED_APPLY_DIRICHLET)
    ref = _oracle(m, q, "diffusion", x, k=k.reshape(m.n_elem, -1), mask=m.boundary)
    assert rel_err(y, ref) <= 1e-12
    b = m.boundary.astype(bool)
    np.testing.assert_array_equal(y[b], x[b])
    nt.close()


def test_single_element_and_constant_coefficient(ceed):
    # one element (a block of 32 lanes with 31 idle), k = 2.5 constant
    m = synthetic.TetMesh(1, 1, 1, 3, seed=0)
    sel = np.array([4])
    dofs = m.elem_dofs[sel]
    uniq, local = np.unique(dofs, return_inverse=True)
    dofs1 = local.reshape(dofs.shape).astype(np.int32)
    interp, grad, qw, qref = ceed.ceed_simplex_basis(3, 4)
    nt = ceed.ceed_nt_setup(1, len(uniq), interp, grad, qw, qref, torch.from_numpy(dofs1).cuda(),
                            torch.from_numpy(np.ascontiguousarray(m.vertices[sel])).cuda())
    qd = _qdata(ceed, nt, "diffusion", ceed.CEED_F64, ceed.CEED_COEFF_CONST, 2.5)
    x = synthetic.uniform(len(uniq), seed=1)
    y = _apply(ceed, nt, "diffusion", qd, ceed.CEED_F64, x)
    sp_ = sx.SimplexSpace(3, 4)
    ref = fem.apply(sp_, dofs1, 2.5 * sx.qdata_diffusion(sp_, m.vertices[sel]), x, fem.DIFFUSION)
    assert rel_err(y, ref) <= 1e-12
    nt.close()


def test_autotune_keeps_a_valid_choice(ceed):
    p, q = 3, 4
    m = synthetic.TetMesh(4, 4, 3, p, seed=2)
    nt = _setup(ceed, m, q)
    qd = _qdata(ceed, nt, "diffusion", ceed.CEED_F64)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=3)).cuda()
    y = torch.empty_like(x)
    algo, eta, mode, ms = ceed.ceed_nt_autotune(nt, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F64, x, y)
    assert algo in (ceed.CEED_NT_FUSED, ceed.CEED_NT_GEMM) and ms > 0
    yv = _apply(ceed, nt, "diffusion", qd, ceed.CEED_F64, x.cpu().numpy())
    assert rel_err(yv, _oracle(m, q, "diffusion", x.cpu().numpy())) <= 1e-12
    nt.close()


def test_invalid_arguments(ceed):
    m = synthetic.TetMesh(1, 1, 1, 1, seed=0)
    bad = m.elem_dofs.copy()
    bad[0, 0] = m.n_ldof + 5
    interp, grad, qw, qref = ceed.ceed_simplex_basis(1, 2)
    with pytest.raises(ceed.CeedError):
        ceed.ceed_nt_setup(m.n_elem, m.n_ldof, interp, grad, qw, qref, torch.from_numpy(bad).cuda(),
                           torch.from_numpy(m.vertices).cuda())
    # inverted element: det J < 0 is reported at the quadrature-data build
    V = m.vertices.copy()
    V[0, [1, 2]] = V[0, [2, 1]]
    nt = ceed.ceed_nt_setup(m.n_elem, m.n_ldof, interp, grad, qw, qref, torch.from_numpy(m.elem_dofs).cuda(),
                            torch.from_numpy(V).cuda())
    qd = ceed.alloc_nt_qdata(nt, ceed.CEED_OP_MASS, ceed.CEED_F64)
    with pytest.raises(ceed.CeedError) as ei:
        ceed.ceed_nt_build_qdata(nt, ceed.CEED_OP_MASS, ceed.CEED_COEFF_ONE, None, ceed.CEED_F64, qd)
    assert ei.value.status == ceed.CEED_ERR_BAD_GEOMETRY
    with pytest.raises(ceed.CeedError):
        ceed.ceed_nt_set_algorithm(nt, ceed.CEED_OP_MASS, ceed.CEED_F64, ceed.CEED_NT_GEMM, 0, 2)  # TF32 needs F32
    with pytest.raises(ceed.CeedError):
        ceed.ceed_nt_set_algorithm(nt, ceed.CEED_OP_MASS, ceed.CEED_F64, ceed.CEED_NT_TC)  # tensor cores: F32
    nt.close()


def _sampled_oracle(m, q, x, nodes):
    """Oracle y at the given nodes only: dense actions of the elements that contain them."""
    hit = np.isin(m.elem_dofs, nodes).any(1)
    els = np.nonzero(hit)[0]
    sp_ = sx.SimplexSpace(m.p, q)
    qd = sx.qdata_diffusion(sp_, m.vertices[els], "sine")
    Ye = fem.element_action(sp_, x[m.elem_dofs[els]], qd, fem.DIFFUSION)
    y = np.zeros(m.n_ldof)
    np.add.at(y, m.elem_dofs[els].reshape(-1), Ye.reshape(-1))
    return y[nodes]


@pytest.mark.parametrize("algo,prec,mode,tol", [("fused", "f64", 0, 1e-12), ("gemm", "f64", 1, 1e-12),
                                                ("fused", "f32", 0, 2e-5), ("tc", "f32", 0, 2e-5)])
def test_full_size_sampled(ceed, algo, prec, mode, tol):
    # the benchmark's tetrahedral workload (48^3 cubes x 6 = 663,552 degree-4 elements, 7.1M nodes),
    # compared with the oracle on 400 sampled nodes
    p, q = 4, 5
    m = synthetic.TetMesh(48, 48, 48, p, seed=0)
    nt = _setup(ceed, m, q, dirichlet=False)
    cprec = ceed.CEED_F64 if prec == "f64" else ceed.CEED_F32
    qd = _qdata(ceed, nt, "diffusion", cprec)
    if algo == "gemm":
        ceed.ceed_nt_set_algorithm(nt, ceed.CEED_OP_DIFFUSION, cprec, ceed.CEED_NT_GEMM, 0, mode)
    elif algo == "tc":
        ceed.ceed_nt_set_algorithm(nt, ceed.CEED_OP_DIFFUSION, cprec, ceed.CEED_NT_TC)
    x = synthetic.uniform(m.n_ldof, seed=1)
    y = _apply(ceed, nt, "diffusion", qd, cprec, x)
    ceed.ceed_nt_status(nt)
    nodes = np.random.default_rng(0).choice(m.n_ldof, 400, replace=False)
    ref = _sampled_oracle(m, q, x, nodes)
    assert rel_err(y[nodes], ref) <= tol
    nt.close()
    del qd
    torch.cuda.empty_cache()

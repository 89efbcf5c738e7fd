"""GPU parity of the brick kernel (2 x 2 x 1 element groups of a structured lattice, one thread block
per group: Section 2's gather and scatter done once per group node) against the CPU oracle and the
element kernel.

Tolerance: the brick kernel runs the FP32-pipe operators, so it is held to the same bound as the
element kernel's FP32 paths against the FP64 oracle (c * P * eps32, c = 64, eps32 = 2^-24; BF16 and
FP16 storage add their own quadrature-data rounding), and to the same bound against the element
kernel (the two differ only in the order of the additions at shared nodes).  Repeated applies are
bitwise identical (fixed summation order, no atomics).
"""
import numpy as np
import pytest

import synthetic
from oracle import fem
from _util import gpu_mesh, oracle_qdata, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ceed():
    import paper_2109_05072_gb300 as c
    assert torch.cuda.is_available()
    return c


def _qdata(ceed, mesh, cop, prec):
    qd = ceed.alloc_qdata(mesh, cop, prec)
    ceed.ceed_build_qdata(mesh, cop, ceed.CEED_COEFF_SINE, None, prec, qd)
    return qd


def _run(ceed, mesh, cop, qd, prec, x, flags=0):
    y = torch.empty_like(x)
    f = ceed.ceed_apply_diffusion if cop == ceed.CEED_OP_DIFFUSION else ceed.ceed_apply_mass
    f(mesh, qd, prec, x, y, flags=flags)
    torch.cuda.synchronize()
    return y


def _variant(ceed, mesh, cop, prec, stage):
    ceed.ceed_set_apply_variant(mesh, cop, prec, 0 if stage < 2 else 1, stage)


def test_brick_detection(ceed):
    # even element counts along x and y: one brick per 2 x 2 x 1 cell; odd counts along x or y, or a
    # non-lattice numbering: none
    m = synthetic.HexMesh(4, 2, 3, 3, seed=1)
    mesh = gpu_mesh(ceed, m)
    assert ceed.ceed_mesh_bricks(mesh) == 2 * 1 * 3
    mesh.close()
    m = synthetic.HexMesh(5, 2, 2, 3, seed=1)
    mesh = gpu_mesh(ceed, m)
    assert ceed.ceed_mesh_bricks(mesh) == 0
    with pytest.raises(ceed.CeedError):
        ceed.ceed_set_apply_variant(mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32, 1, 2)
    mesh.close()
    # elements listed in a shuffled order: still a lattice of bricks
    m = synthetic.HexMesh(2, 4, 2, 2, seed=1)
    perm = np.random.default_rng(5).permutation(m.n_elem)
    m.elem_dofs = np.ascontiguousarray(m.elem_dofs[perm])
    m.vertices = np.ascontiguousarray(m.vertices[perm])
    mesh = gpu_mesh(ceed, m)
    assert ceed.ceed_mesh_bricks(mesh) == 1 * 2 * 2
    mesh.close()
    # two nodes swapped in the numbering: not an affine lattice any more
    m = synthetic.HexMesh(2, 2, 2, 2, seed=1)
    swap = np.arange(m.n_ldof)
    swap[[3, 7]] = swap[[7, 3]]
    m.elem_dofs = np.ascontiguousarray(swap[m.elem_dofs].astype(np.int32))
    mesh = gpu_mesh(ceed, m, dirichlet=False)
    assert ceed.ceed_mesh_bricks(mesh) == 0
    mesh.close()


# FP32 (1), BF16 (2), FP16 (3) quadrature data and on-the-fly geometry (4), every p, both rules
BRICK_CASES = [(p, q, op, prec) for p in range(1, 9) for q in ("gll", "gauss") for op in ("diffusion", "mass")
               for prec in (1,)] + [(7, "gll", "diffusion", 2), (7, "gll", "diffusion", 3), (7, "gll", "diffusion", 4),
                                    (3, "gauss", "diffusion", 4), (4, "gll", "mass", 2)]


def _bound(prec, P):
    return {1: 64 * P * EPS32, 2: 2e-2, 3: 2e-3, 4: 64 * P * EPS32}[prec]


@pytest.mark.parametrize("p,qkind,op,prec", BRICK_CASES)
def test_brick_matches_oracle_and_element_kernel(ceed, p, qkind, op, prec):
    # several bricks per colour, bricks on every side of a brick (the 6 x 4 x 3 lattice at low order)
    dims = (6, 4, 3) if p <= 3 else (4, 4, 2)
    m = synthetic.HexMesh(*dims, p, seed=20 + p)
    mesh = gpu_mesh(ceed, m, qkind)
    assert ceed.ceed_mesh_bricks(mesh) == dims[0] * dims[1] * dims[2] // 4
    cop = ceed.CEED_OP_DIFFUSION if op == "diffusion" else ceed.CEED_OP_MASS
    qd = _qdata(ceed, mesh, cop, prec)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=21)).cuda()
    _variant(ceed, mesh, cop, prec, 1)
    y_elem = _run(ceed, mesh, cop, qd, prec, x)
    sp_, qref = oracle_qdata(m, qkind, op, "sine")
    ref = fem.apply(sp_, m.elem_dofs, qref, x.cpu().numpy(), fem.DIFFUSION if op == "diffusion" else fem.MASS)
    bound = _bound(prec, p + 1)
    ran = 0
    for stage in (2, 3):
        _variant(ceed, mesh, cop, prec, stage)
        try:
            y = _run(ceed, mesh, cop, qd, prec, x)
        except ceed.CeedError as ex:  # staged bricks of the largest orders exceed the shared memory
            assert stage == 3 and p >= 7, str(ex)
            continue
        ran += 1
        err = rel_err(y.cpu().numpy(), ref)
        print(f"brick stage {stage} p={p} {qkind} {op} prec {prec}: rel err vs FP64 oracle {err:.3e}")
        assert err <= bound
        assert rel_err(y.cpu().numpy(), y_elem.cpu().numpy()) <= bound
        assert torch.equal(_run(ceed, mesh, cop, qd, prec, x), y)   # deterministic
    assert ran >= 1
    mesh.close()


@pytest.mark.parametrize("p,qkind", [(7, "gll"), (2, "gauss"), (4, "gll")])
def test_brick_dirichlet_masked_apply(ceed, p, qkind):
    m = synthetic.HexMesh(4, 2, 3, p, seed=30)
    mesh = gpu_mesh(ceed, m, qkind)
    qd = _qdata(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=31)).cuda()
    sp_, qref = oracle_qdata(m, qkind, "diffusion", "sine")
    Am = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, qref, v, fem.DIFFUSION), m.boundary)
    ref = Am(x.cpu().numpy())
    for stage in (2, 3):
        _variant(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32, stage)
        y = _run(ceed, mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F32, x, flags=ceed.CEED_APPLY_DIRICHLET)
        yn = y.cpu().numpy()
        assert rel_err(yn, ref) <= 64 * (p + 1) * EPS32
        b = m.boundary.astype(bool)
        assert np.array_equal(yn[b], x.cpu().numpy()[b])   # identity rows, exactly
    mesh.close()


def test_brick_autotune_and_several_columns(ceed):
    # the autotuner may choose a brick variant; a multi-column apply then runs the element kernel
    m = synthetic.HexMesh(4, 4, 4, 5, seed=40)
    mesh = gpu_mesh(ceed, m, "gll")
    cop, prec = ceed.CEED_OP_DIFFUSION, ceed.CEED_F32
    qd = _qdata(ceed, mesh, cop, prec)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=41)).cuda()
    ne, stage, ms = ceed.ceed_autotune_apply(mesh, cop, qd, prec, x, torch.empty_like(x))
    assert stage in (0, 1, 2, 3) and ms > 0
    sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
    ref = fem.apply(sp_, m.elem_dofs, qref, x.cpu().numpy(), fem.DIFFUSION)
    assert rel_err(_run(ceed, mesh, cop, qd, prec, x).cpu().numpy(), ref) <= 64 * 6 * EPS32
    _variant(ceed, mesh, cop, prec, 2)
    x2 = torch.from_numpy(synthetic.uniform(2 * m.n_ldof, seed=42)).cuda()
    y2 = torch.empty_like(x2)
    ceed.ceed_apply_diffusion(mesh, qd, prec, x2, y2, nrhs=2)
    torch.cuda.synchronize()
    X = x2.cpu().numpy().reshape(m.n_ldof, 2)
    Y = y2.cpu().numpy().reshape(m.n_ldof, 2)
    for c in range(2):
        ref = fem.apply(sp_, m.elem_dofs, qref, np.ascontiguousarray(X[:, c]), fem.DIFFUSION)
        assert rel_err(Y[:, c], ref) <= 64 * 6 * EPS32
    mesh.close()


def test_brick_cg_separate_kernels(ceed):
    # mixed-precision CG (reliable updates) whose FP32 operator runs the brick kernel (one kernel per
    # CG step), and the fused iteration (element kernel): both reach the FP64 residual target
    m = synthetic.HexMesh(4, 4, 4, 4, seed=50)
    mesh = gpu_mesh(ceed, m, "gll")
    q64 = _qdata(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F64)
    q32 = _qdata(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    _variant(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32, 2)
    b = torch.empty(m.n_ldof, dtype=torch.float64, device="cuda")
    ceed.ceed_manufactured_rhs(mesh, ceed.CEED_COEFF_SINE, b, flags=ceed.CEED_APPLY_DIRICHLET)
    xs = []
    for sep in (1, 0):
        x = torch.empty_like(b)
        st, rep = ceed.ceed_cg_solve(mesh, q64, ceed.CEED_F64, b, x, mode=ceed.CEED_CG_MIXED_RELIABLE, tol=1e-10,
                                     max_iter=2000, op=ceed.CEED_OP_DIFFUSION, qdata_lo=q32,
                                     prec_lo=ceed.CEED_F32, separate_kernels=sep)
        assert rep["rel_residual"] <= 1e-10
        xs.append(x.cpu().numpy())
    assert rel_err(xs[0], xs[1]) <= 1e-8
    mesh.close()


def test_brick_copy_wait_expiry_then_recovery(ceed):
    # the staged brick variant waits (bounded) for its quadrature-data copies: with the wait limit at
    # zero it gives up at once, writes nothing, reports CEED_ERR_TIMEOUT and leaves no hung GPU;
    # the next apply with the default limit is correct
    m = synthetic.HexMesh(4, 2, 3, 3, seed=60)
    mesh = gpu_mesh(ceed, m, "gll")
    qd = _qdata(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32)
    x = torch.from_numpy(synthetic.uniform(m.n_ldof, seed=61)).cuda()
    _variant(ceed, mesh, ceed.CEED_OP_DIFFUSION, ceed.CEED_F32, 3)
    y = torch.zeros_like(x)
    ceed.ceed_set_wait_limits(0, -1)
    try:
        ceed.ceed_apply_diffusion(mesh, qd, ceed.CEED_F32, x, y)
        with pytest.raises(ceed.CeedError) as ei:
            ceed.ceed_mesh_status(mesh)
        assert ei.value.status == ceed.CEED_ERR_TIMEOUT
    finally:
        ceed.ceed_set_wait_limits(-1, -1)
    ceed.ceed_mesh_status(mesh)
    y = _run(ceed, mesh, ceed.CEED_OP_DIFFUSION, qd, ceed.CEED_F32, x)
    ceed.ceed_mesh_status(mesh)
    sp_, qref = oracle_qdata(m, "gll", "diffusion", "sine")
    ref = fem.apply(sp_, m.elem_dofs, qref, x.cpu().numpy(), fem.DIFFUSION)
    assert rel_err(y.cpu().numpy(), ref) <= 64 * 4 * EPS32
    mesh.close()

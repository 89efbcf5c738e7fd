"""Pins for the oracle's PCG, manufactured solution and adjoint (Section 1: CG on the matrix-free operator)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem


def _problem(N, p, seed=0, coeff="sine", perturb=0.1):
    m = synthetic.cube_mesh(N, p, seed=seed, perturb=perturb)
    sp_ = fem.Space(p, "gll")
    G = fem.qdata_diffusion(sp_, m.vertices, "sine" if coeff == "sine" else None)
    A = fem.assemble(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof)
    mask = m.boundary.astype(bool)
    Am = A.tolil()
    Am[mask, :] = 0
    Am[:, mask] = 0
    Am = Am.tocsr()
    Am = Am + __import__("scipy.sparse", fromlist=["diags"]).diags(mask.astype(float))
    b = fem.manufactured_rhs(sp_, m.vertices, m.elem_dofs, m.n_ldof, coeff, mask=mask)
    d = fem.jacobi_diagonal(sp_, m.elem_dofs, G, fem.DIFFUSION, m.n_ldof, mask=mask)
    return m, sp_, G, Am, b, d


def test_pcg_matches_direct_solve():
    m, sp_, G, Am, b, d = _problem(3, 3)
    x, it, rel, hist = fem.pcg(lambda v: Am @ v, b, 1.0 / d, tol=1e-12, maxit=2000)
    xd = spla.spsolve(Am.tocsc(), b)
    assert rel <= 1e-12 and it < 2000
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-10 * np.abs(xd).max())
    assert np.linalg.norm(b - Am @ x) <= 2e-12 * np.linalg.norm(b)
    # the matrix-free masked operator is the same operator
    Amf = fem.masked(lambda v: fem.apply(sp_, m.elem_dofs, G, v, fem.DIFFUSION), m.boundary)
    np.testing.assert_allclose(Amf(x), Am @ x, atol=1e-13)


def test_pcg_exact_in_n_steps_small():
    # CG in exact arithmetic terminates in at most n steps; on a 2x2 SPD system it is exact in 2
    A = np.array([[4.0, 1.0], [1.0, 3.0]])
    b = np.array([1.0, 2.0])
    x, it, rel, _ = fem.pcg(lambda v: A @ v, b, np.ones(2), tol=1e-15, maxit=10)
    assert it <= 2
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-14)


def test_reliable_pcg_with_exact_operator_is_pcg():
    # with apply_lo = apply_hi the replaced residual equals the recurrence one up to rounding, so the
    # reliable-update run takes the ordinary PCG iterates
    m, sp_, G, Am, b, d = _problem(3, 3)
    A = lambda v: Am @ v
    x0, it0, _, _ = fem.pcg(A, b, 1.0 / d, tol=1e-10, maxit=2000)
    x1, it1, rel1, evals = fem.pcg_reliable(A, A, b, 1.0 / d, tol=1e-10, delta=0.1)
    assert rel1 <= 1e-10 and evals >= 10
    assert abs(it1 - it0) <= 1
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-9 * np.abs(x0).max())


def test_reliable_pcg_recovers_fp64_accuracy_from_a_perturbed_operator():
    # the inner operator carries relative errors of 1e-6 in its entries (far coarser than FP32
    # rounding of the matrix-free operator): plain PCG on it stalls near the perturbation level in
    # the true residual, residual replacement reaches 1e-10 in about the exact iteration count
    m, sp_, G, Am, b, d = _problem(3, 4)
    rng = np.random.default_rng(5)
    E = Am.copy()
    E.data = E.data * (1.0 + 1e-6 * rng.uniform(-1, 1, size=E.data.size))
    E = 0.5 * (E + E.T)
    lo, hi = (lambda v: E @ v), (lambda v: Am @ v)
    _, it_exact, _, _ = fem.pcg(hi, b, 1.0 / d, tol=1e-10, maxit=5000)
    x_plain, _, _, _ = fem.pcg(lo, b, 1.0 / d, tol=1e-12, maxit=5000)
    plain_true = np.linalg.norm(b - Am @ x_plain) / np.linalg.norm(b)
    x, it, rel, evals = fem.pcg_reliable(lo, hi, b, 1.0 / d, tol=1e-10, delta=0.1)
    assert plain_true > 1e-9
    assert rel <= 1e-10 and np.linalg.norm(b - Am @ x) <= 1e-10 * np.linalg.norm(b)
    assert it <= 1.25 * it_exact + 5, (it, it_exact)
    assert evals >= 3

def test_manufactured_source_closed_form():
    # f = -div(k grad u*) checked against a finite-difference divergence of k grad u* at a few points
    rng = np.random.default_rng(0)
    X = rng.uniform(0.1, 0.9, (5, 3))
    h = 1e-4

    def flux(Y):
        k = fem.coeff_sine(Y)
        g = np.zeros_like(Y)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            g[:, d] = (fem.exact_solution(Y + e) - fem.exact_solution(Y - e)) / (2 * h)
        return k[:, None] * g
    div = np.zeros(len(X))
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        div += (flux(X + e)[:, d] - flux(X - e)[:, d]) / (2 * h)
    np.testing.assert_allclose(fem.manufactured_source(X), -div, rtol=1e-5)


@pytest.mark.parametrize("p,Ns", [(1, (4, 8, 16)), (2, (4, 8, 12)), (3, (4, 6, 8)), (4, (2, 4, 6))])
def test_convergence_order(p, Ns):
    # O(h^{p+1}) L2 convergence of the discrete solution to u* (Section 1, p-th order approximations).
    # Even N only (odd N changes how the element edges sit against the sine's extrema); on these coarse
    # meshes the fitted slope sits at or slightly above p+1 (pre-asymptotic), so the window is [p+0.7, p+1.6].
    # A dropped term or wrong quadrature/geometry factor makes the solution converge at <= p or not at all.
    errs, hs = [], []
    for N in Ns:
        m, sp_, G, Am, b, d = _problem(N, p, seed=N)
        x, it, rel, _ = fem.pcg(lambda v: Am @ v, b, 1.0 / d, tol=1e-12, maxit=5000)
        assert rel <= 1e-12
        errs.append(fem.l2_error(p, m.vertices, m.elem_dofs, x))
        hs.append(1.0 / N)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert p + 0.7 <= slope <= p + 1.6, (slope, errs)
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:]))


def test_adjoint_gradient_fd():
    # L = 0.5 ||A(k) x - b||^2, directional central differences in k and in x
    p = 2
    m = synthetic.cube_mesh(2, p, seed=1)
    sp_ = fem.Space(p, "gll")
    k = synthetic.lognormal(m.n_elem * sp_.nq, seed=2).reshape(m.n_elem, sp_.nq)
    x = synthetic.uniform(m.n_ldof, seed=3)
    b = synthetic.uniform(m.n_ldof, seed=4)
    L, gx, gk = fem.adjoint(sp_, m.vertices, m.elem_dofs, k, x, b)
    vk = synthetic.uniform(k.size, seed=5).reshape(k.shape)
    vx = synthetic.uniform(m.n_ldof, seed=6)
    hk = 1e-6 * np.abs(k).max() / np.abs(vk).max()
    Lp = fem.adjoint(sp_, m.vertices, m.elem_dofs, k + hk * vk, x, b)[0]
    Lm = fem.adjoint(sp_, m.vertices, m.elem_dofs, k - hk * vk, x, b)[0]
    assert abs((Lp - Lm) / (2 * hk) - np.sum(gk * vk)) < 1e-6 * abs(np.sum(gk * vk))
    hx = 1e-6
    Lp = fem.adjoint(sp_, m.vertices, m.elem_dofs, k, x + hx * vx, b)[0]
    Lm = fem.adjoint(sp_, m.vertices, m.elem_dofs, k, x - hx * vx, b)[0]
    assert abs((Lp - Lm) / (2 * hx) - gx @ vx) < 1e-6 * abs(gx @ vx)


def test_adjoint_per_entry_fd_and_identity():
    p = 1
    m = synthetic.cube_mesh(1, p, seed=0)
    sp_ = fem.Space(p, "gll")
    k = synthetic.lognormal(sp_.nq, seed=7).reshape(1, sp_.nq)
    x = synthetic.uniform(m.n_ldof, seed=8)
    b = synthetic.uniform(m.n_ldof, seed=9)
    L, gx, gk = fem.adjoint(sp_, m.vertices, m.elem_dofs, k, x, b)
    for q in range(sp_.nq):
        dk = np.zeros_like(k)
        dk[0, q] = 1e-6
        fd = (fem.adjoint(sp_, m.vertices, m.elem_dofs, k + dk, x, b)[0]
              - fem.adjoint(sp_, m.vertices, m.elem_dofs, k - dk, x, b)[0]) / 2e-6
        assert abs(fd - gk[0, q]) < 1e-6 * max(1.0, abs(gk[0, q]))
    # <dL/dx, v> = <r, A v>
    G = fem.qdata_diffusion(sp_, m.vertices, k)
    A = lambda v: fem.apply(sp_, m.elem_dofs, G, v, fem.DIFFUSION)
    r = A(x) - b
    v = synthetic.uniform(m.n_ldof, seed=10)
    assert abs(gx @ v - r @ A(v)) < 1e-13 * abs(r @ A(v))

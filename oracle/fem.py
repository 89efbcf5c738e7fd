"""Dense (no sum factorization) finite-element operators for the oracle.

Test infrastructure only.  Each function states the passage of the paper (or
the reading of it) that it follows.  Index conventions shared with the C-ABI:
  element nodes  n = a + P (b + P c)       (a along r, fastest)
  quad points    q = i + Q (j + Q k)       (i along r, fastest)
  per-element arrays [E, nq] are in the caller's element order.
Geometry arguments (named `vertices`) are either the trilinear vertices [E, 8, 3]
or an Isoparametric (curved, degree-p) element geometry.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import gauss, gll, lagrange, rule

MASS = "mass"
DIFFUSION = "diffusion"


class Space:
    """Reference Q_p hexahedron with a tensor quadrature rule.

    Q_p Lagrange basis on the p+1 Gauss-Lobatto points per direction (Section 1);
    quadrature either collocated on the same GLL points (BP5: 'gll', Q = p+1)
    or Gauss (BP1/BP3: 'gauss', default Q = p+2).  The basis is tabulated at
    every 3D quadrature point as the product of the three 1D Lagrange values:
    Phi[q, n] = l_a(r_i) l_b(s_j) l_c(t_k), and the reference gradient
    dPhi[d, q, n] differentiates the factor for direction d.
    """

    def __init__(self, p: int, qkind: str = "gll", Q: int | None = None):
        if p < 1:
            raise ValueError("p >= 1")
        self.p, self.P = p, p + 1
        if Q is None:
            Q = self.P if qkind == "gll" else p + 2
        self.qkind, self.Q = qkind, Q
        self.nodes, self.node_w = gll(self.P)
        self.xq, self.wq = rule(qkind, Q)
        self.nd, self.nq = self.P ** 3, Q ** 3
        self.Phi, self.dPhi, self.W, self.XI = tabulate(self.nodes, self.xq, self.wq)


def tabulate(nodes, xq, wq):
    """Phi [nq, nd], dPhi [3, nq, nd], weights W [nq], reference points XI [nq, 3]."""
    P, Q = len(nodes), len(xq)
    L, dL = lagrange(nodes, xq)                      # [Q, P]
    # axes (k, j, i, c, b, a): point (r_i, s_j, t_k), node (a, b, c)
    Lr, Ls, Lt = L[None, None, :, None, None, :], L[None, :, None, None, :, None], L[:, None, None, :, None, None]
    dLr, dLs, dLt = dL[None, None, :, None, None, :], dL[None, :, None, None, :, None], dL[:, None, None, :, None, None]
    Phi = (Lr * Ls * Lt).reshape(Q ** 3, P ** 3)
    dPhi = np.stack([(dLr * Ls * Lt).reshape(Q ** 3, P ** 3),
                     (Lr * dLs * Lt).reshape(Q ** 3, P ** 3),
                     (Lr * Ls * dLt).reshape(Q ** 3, P ** 3)])
    W = (wq[None, None, :] * wq[None, :, None] * wq[:, None, None]).reshape(-1)
    XI = np.stack(np.broadcast_arrays(xq[None, None, :], xq[None, :, None], xq[:, None, None]), -1).reshape(-1, 3)
    return Phi, dPhi, W, XI


def trilinear_map(vertices, XI):
    """Physical points X [E, nq, 3] and Jacobians J [E, nq, 3, 3], J[..., a, b] = dx_a / dxi_b.

    The element map x(r) of Section 1 is read as the trilinear (Q1) map from the
    hexahedron's 8 vertices (local vertex v = vx + 2 vy + 4 vz):
      x(xi) = sum_v N_v(xi) X_v,  N_v = prod_d (1 + s_vd xi_d) / 2,  s_vd = +-1.
    """
    vertices = np.asarray(vertices, dtype=np.float64)
    nq = XI.shape[0]
    N = np.ones((nq, 8))
    dN = np.zeros((nq, 8, 3))
    for v in range(8):
        s = [2.0 * ((v >> d) & 1) - 1.0 for d in range(3)]
        f = [(1.0 + s[d] * XI[:, d]) / 2.0 for d in range(3)]
        N[:, v] = f[0] * f[1] * f[2]
        dN[:, v, 0] = s[0] / 2.0 * f[1] * f[2]
        dN[:, v, 1] = f[0] * s[1] / 2.0 * f[2]
        dN[:, v, 2] = f[0] * f[1] * s[2] / 2.0
    X = np.einsum("qv,evc->eqc", N, vertices)
    J = np.einsum("qvb,eva->eqab", dN, vertices)
    return X, J


class Isoparametric:
    """Curved element geometry of degree p (isoparametric): x(xi) = sum_n phi_n(xi) x_n.

    The element map is interpolated with the element's own Q_p basis from the physical
    positions of its nodes, coords [E, (p+1)^3, 3] in element-node order; Section 2 asks only
    for deformed (non-affine) elements, and this is the usual curved generalisation of the
    trilinear map (same basis for geometry and solution).
    """

    def __init__(self, coords):
        self.coords = np.asarray(coords, dtype=np.float64)


def node_points(p: int, vertices):
    """Physical positions [E, (p+1)^3, 3] of the Q_p element nodes under the trilinear map."""
    nodes, w = gll(p + 1)
    _, _, _, XI = tabulate(nodes, nodes, w)
    X, _ = trilinear_map(vertices, XI)
    return X


def global_node_points(p: int, vertices, elem_dofs, n: int):
    """Positions [n, 3] of the global nodes under the (conforming) trilinear element maps."""
    X = node_points(p, vertices)
    out = np.zeros((n, 3))
    out[np.asarray(elem_dofs).reshape(-1)] = X.reshape(-1, 3)
    return out


def isoparametric_map(space: Space, coords):
    """X [E, nq, 3] and J [E, nq, 3, 3] (J[..., a, b] = dx_a / dxi_b) of the isoparametric map."""
    coords = np.asarray(coords, dtype=np.float64)
    if coords.shape[1] != space.nd:
        raise ValueError("coords must hold the (p+1)^3 nodes of each element")
    X = np.einsum("qn,enc->eqc", space.Phi, coords)
    J = np.einsum("bqn,ena->eqab", space.dPhi, coords)
    return X, J


def element_map(space: Space, geom):
    """(X, J) at the quadrature points: trilinear from vertices [E, 8, 3], or isoparametric."""
    if isinstance(geom, Isoparametric):
        return isoparametric_map(space, geom.coords)
    return trilinear_map(geom, space.XI)


def coeff_sine(X):
    """k(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) at points X [..., 3]."""
    s = np.sin(2.0 * np.pi * X)
    return 1.0 + 0.5 * s[..., 0] * s[..., 1] * s[..., 2]


def qdata_mass(space: Space, vertices, rho=None):
    """Mass quadrature data w_q |det J_q| rho_q, [E, nq]."""
    _, J = element_map(space, vertices)
    qd = space.W[None, :] * np.abs(np.linalg.det(J))
    if rho is not None:
        qd = qd * rho
    return qd


def geometric_factor(space: Space, vertices):
    """w_q |det J| J^{-1} J^{-T} per point, [E, nq, 3, 3] (the symmetric G^e of Section 2 without k)."""
    _, J = element_map(space, vertices)
    Jinv = np.linalg.inv(J)
    return (space.W[None, :] * np.abs(np.linalg.det(J)))[..., None, None] * (Jinv @ np.swapaxes(Jinv, -1, -2))


def qdata_diffusion(space: Space, vertices, k=None):
    """Diffusion quadrature data G_q = k_q w_q |det J| J^{-1} J^{-T}, [E, nq, 3, 3].

    The six distinct entries are the diagonal matrices G_rr ... G_tt of the
    symmetric tensor G^e in A^e = D^T G^e D (Section 2).  k: None (k = 1),
    the string 'sine' (coeff_sine at the physical points) or an [E, nq] array.
    """
    G = geometric_factor(space, vertices)
    if k is None:
        return G
    if isinstance(k, str):
        if k != "sine":
            raise ValueError(k)
        X, _ = element_map(space, vertices)
        k = coeff_sine(X)
    return np.asarray(k)[..., None, None] * G


def element_action(space: Space, U, qd, op: str):
    """Dense per-element action y^e = B^T D B u^e for U [e, nd] (or [e, nd, m])."""
    squeeze = U.ndim == 2
    if squeeze:
        U = U[..., None]
    if op == MASS:
        uq = np.einsum("qn,enm->eqm", space.Phi, U)
        Y = np.einsum("qn,eqm->enm", space.Phi, qd[..., None] * uq)
    elif op == DIFFUSION:
        g = np.einsum("dqn,enm->edqm", space.dPhi, U)
        v = np.einsum("eqab,ebqm->eaqm", qd, g)
        Y = np.einsum("dqn,edqm->enm", space.dPhi, v)
    else:
        raise ValueError(op)
    return Y[..., 0] if squeeze else Y


def apply(space: Space, elem_dofs, qd, x, op: str, chunk: int = 256):
    """y = sum_e P_e^T A^e P_e x: dense element actions, scatter-add in element order.

    x is [n] or [n, m] (m independent columns: components or right-hand sides,
    A (x) I).  qd is [E, nq] (mass) or [E, nq, 3, 3] (diffusion).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    E = elem_dofs.shape[0]
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        idx = elem_dofs[e0:e1]
        Ye = element_action(space, x[idx], qd[e0:e1], op)
        np.add.at(y, idx.reshape(-1), Ye.reshape((-1,) + x.shape[1:]))
    return y


def element_matrices(space: Space, qd, op: str):
    """Dense A^e [E, nd, nd] (tiny meshes only)."""
    if op == MASS:
        return np.einsum("qn,eq,qm->enm", space.Phi, qd, space.Phi)
    return np.einsum("aqn,eqab,bqm->enm", space.dPhi, qd, space.dPhi)


def assemble(space: Space, elem_dofs, qd, op: str, n: int):
    """Assembled sparse A = sum_e P_e^T A^e P_e (CSR), the full-assembly comparison of Section 2."""
    Ae = element_matrices(space, qd, op)
    rows = np.repeat(elem_dofs[:, :, None], space.nd, axis=2)
    cols = np.repeat(elem_dofs[:, None, :], space.nd, axis=1)
    return sp.coo_matrix((Ae.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n)).tocsr()


def masked(apply_fn, mask):
    """Operator with homogeneous Dirichlet rows/columns replaced by the identity."""
    m = np.asarray(mask).astype(bool)

    def f(x):
        xi = np.where(m if x.ndim == 1 else m[:, None], 0.0, x)
        y = apply_fn(xi)
        return np.where(m if x.ndim == 1 else m[:, None], x, y)
    return f


def jacobi_diagonal(space: Space, elem_dofs, qd, op: str, n: int, mask=None):
    """diag(A) = sum_e P_e^T diag(A^e); 1 on Dirichlet nodes when a mask is given."""
    if op == MASS:
        de = np.einsum("qn,eq->en", space.Phi ** 2, qd)
    else:
        de = np.einsum("aqn,eqab,bqn->en", space.dPhi, qd, space.dPhi)
    d = np.zeros(n)
    np.add.at(d, elem_dofs.reshape(-1), de.reshape(-1))
    if mask is not None:
        d[np.asarray(mask).astype(bool)] = 1.0
    return d


def pcg(apply_fn, b, dinv, tol: float = 1e-10, maxit: int = 10000, x0=None):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), the outer solver of Section 1.

    Stops when ||r||_2 <= tol ||b||_2 on the recurrence residual.  Returns
    (x, iterations, relative recurrence residual, history of relative residuals).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_fn(x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / nb]
    it = 0
    while it < maxit and hist[-1] > tol:
        q = apply_fn(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist[-1], np.array(hist)


def pcg_reliable(apply_lo, apply_hi, b, dinv, tol: float = 1e-10, delta: float = 0.1, maxit: int = 10000):
    """PCG run with an inexact operator `apply_lo` and reliable updates (Sleijpen and van der Vorst,
    "Reliable updated residuals in hybrid Bi-CG methods", Computing 56, 1996): the reading of the
    mixed-precision CG of Section 1's solver in which the Krylov process is never restarted.

    The recurrence residual follows apply_lo; each time its norm has fallen by `delta` since the
    last replacement (or has reached the tolerance), the true residual b - apply_hi(x) is computed,
    the run stops if it meets tol, and otherwise it replaces the recurrence residual before the
    step's beta: z = D^{-1} r and beta = r.z / r.z_old come from the true residual, and the new
    direction p = z + beta p continues the same Krylov process.  x0 = 0.  Returns (x, iterations,
    true relative residual, number of true-residual evaluations).
    """
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    ref = np.linalg.norm(r)
    evals, it = 1, 0
    true_rel = ref / nb
    while it < maxit and true_rel > tol:
        q = apply_lo(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        nr = np.linalg.norm(r)
        if nr <= tol * nb or nr <= delta * ref:
            r = b - apply_hi(x)
            evals += 1
            true_rel = np.linalg.norm(r) / nb
            ref = np.linalg.norm(r)
            if true_rel <= tol:
                break
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, true_rel, evals

def exact_solution(X):
    """u*(x) = sin(pi x) sin(pi y) sin(pi z): smooth, zero on the boundary of the unit cube."""
    s = np.sin(np.pi * X)
    return s[..., 0] * s[..., 1] * s[..., 2]


def manufactured_source(X, coeff: str = "sine"):
    """f = -div(k grad u*) in closed form for k = coeff_sine (or k = 1 for coeff='one')."""
    s, c = np.sin(np.pi * X), np.cos(np.pi * X)
    u = s[..., 0] * s[..., 1] * s[..., 2]
    if coeff == "one":
        return 3.0 * np.pi ** 2 * u
    s2, c2 = np.sin(2 * np.pi * X), np.cos(2 * np.pi * X)
    k = 1.0 + 0.5 * s2[..., 0] * s2[..., 1] * s2[..., 2]
    gk = np.pi * np.stack([c2[..., 0] * s2[..., 1] * s2[..., 2],
                           s2[..., 0] * c2[..., 1] * s2[..., 2],
                           s2[..., 0] * s2[..., 1] * c2[..., 2]], -1)
    gu = np.pi * np.stack([c[..., 0] * s[..., 1] * s[..., 2],
                           s[..., 0] * c[..., 1] * s[..., 2],
                           s[..., 0] * s[..., 1] * c[..., 2]], -1)
    return -(gk * gu).sum(-1) + 3.0 * np.pi ** 2 * k * u


def manufactured_rhs(space: Space, vertices, elem_dofs, n: int, coeff: str = "sine", mask=None):
    """b_i = sum_e sum_q w_q |det J| f(x_q) phi_i(x_q), same quadrature as the operator; 0 on Dirichlet nodes."""
    X, J = element_map(space, vertices)
    fq = space.W[None, :] * np.abs(np.linalg.det(J)) * manufactured_source(X, coeff)
    be = np.einsum("qn,eq->en", space.Phi, fq)
    b = np.zeros(n)
    np.add.at(b, elem_dofs.reshape(-1), be.reshape(-1))
    if mask is not None:
        b[np.asarray(mask).astype(bool)] = 0.0
    return b


def l2_error(p: int, vertices, elem_dofs, u, qextra: int = 3):
    """||u_h - u*||_{L2} with Gauss quadrature of p+qextra points per direction."""
    sp_ = Space(p, "gauss", p + qextra)
    X, J = element_map(sp_, vertices)
    uh = np.einsum("qn,en->eq", sp_.Phi, u[elem_dofs])
    err = (uh - exact_solution(X)) ** 2
    return float(np.sqrt(np.sum(sp_.W[None, :] * np.abs(np.linalg.det(J)) * err)))


def adjoint(space: Space, vertices, elem_dofs, k, x, b):
    """Loss L = 0.5 ||A(k) x - b||^2 and its gradients (dL/dx, dL/dk).

    A(k) = sum_e P_e^T D^T G^e(k) D P_e with G_q = k_q Ghat_q and
    Ghat_q = w_q |det J| J^{-1} J^{-T}.  With r = A x - b:
      dL/dx = A^T r = A r (A is symmetric),
      dL/dk_{e,q} = (grad_xi r^e)_q^T Ghat_q (grad_xi x^e)_q.
    """
    Gh = geometric_factor(space, vertices)
    qd = np.asarray(k)[..., None, None] * Gh
    n = len(x)
    r = apply(space, elem_dofs, qd, x, DIFFUSION) - b
    L = 0.5 * float(r @ r)
    dLdx = apply(space, elem_dofs, qd, r, DIFFUSION)
    gr = np.einsum("dqn,en->edq", space.dPhi, r[elem_dofs])
    gx = np.einsum("dqn,en->edq", space.dPhi, x[elem_dofs])
    dLdk = np.einsum("eaq,eqab,ebq->eq", gr, Gh, gx)
    return L, dLdx, dLdk


def cost_model(p: int, collocated: bool = True):
    """Per-element reads and flops of the factored stiffness action (Section 2 preamble).

    Reads: 7 (p+1)^3 (u^e and the six G factors).  Flops: 12 (p+1)^4 + 15 (p+1)^3,
    with the first term doubled for non-collocated quadrature.
    """
    P = p + 1
    return 7 * P ** 3, (12 if collocated else 24) * P ** 4 + 15 * P ** 3


def prolongation_element(p_coarse: int, p_fine: int):
    """Element interpolation matrix [P_f^3, P_c^3]: the coarse Q_{p_c} basis (Lagrange on its GLL nodes)
    evaluated at the fine GLL nodes of the same reference element, as the product of 1D values.

    This is the transfer of p-multigrid between orders on one mesh (the p-multigrid the paper names
    as the usual replacement of low-order preconditioners, Section 1): a coarse finite-element
    function, evaluated at the fine nodes, is the same function in the fine space.
    """
    xc, _ = gll(p_coarse + 1)
    xf, _ = gll(p_fine + 1)
    L, _ = lagrange(xc, xf)                       # [Pf, Pc]
    Pf, Pc = p_fine + 1, p_coarse + 1
    # M[k, j, i, c, b, a] = L[k, c] L[j, b] L[i, a]: fine node (i, j, k), coarse node (a, b, c)
    M = L[:, None, None, :, None, None] * L[None, :, None, None, :, None] * L[None, None, :, None, None, :]
    return M.reshape(Pf ** 3, Pc ** 3)


def prolongate(p_coarse, p_fine, dofs_coarse, dofs_fine, u_coarse, n_fine):
    """u_f = P u_c: interpolate element by element; every element gives the same value at a shared
    fine node (the coarse function is continuous), so the first element in order sets it."""
    M = prolongation_element(p_coarse, p_fine)
    uf = np.full(n_fine, np.nan)
    vals = np.einsum("fc,ec->ef", M, u_coarse[dofs_coarse])
    for e in range(dofs_fine.shape[0]):
        idx = dofs_fine[e]
        new = np.isnan(uf[idx])
        uf[idx[new]] = vals[e][new]
    return uf


def restrict(p_coarse, p_fine, dofs_coarse, dofs_fine, r_fine, n_coarse):
    """r_c = P^T r_f for the assembled interpolation P of `prolongate`: each fine node counted once
    (by the first element in order that contains it)."""
    M = prolongation_element(p_coarse, p_fine)
    w = np.zeros_like(dofs_fine, dtype=np.float64)
    seen = np.zeros(len(r_fine), dtype=bool)
    for e in range(dofs_fine.shape[0]):
        idx = dofs_fine[e]
        first = ~seen[idx]
        w[e][first] = 1.0
        seen[idx] = True
    rc = np.zeros(n_coarse)
    contrib = np.einsum("fc,ef->ec", M, w * r_fine[dofs_fine])
    np.add.at(rc, dofs_coarse.reshape(-1), contrib.reshape(-1))
    return rc

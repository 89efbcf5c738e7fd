"""Non-tensor (tetrahedral) elements for the oracle.  TEST INFRASTRUCTURE ONLY.

Section 3 (libCEED, MAGMA backend): for non-tensor elements the caller supplies the full
interpolation and gradient matrices of the basis at the quadrature points together with the
quadrature weights, and the operator applies them densely, element by element, as
y^e = B^T D B u^e (mass) or G^T D G u^e (diffusion) with the same pointwise D as for hexahedra.
This module gives the degree-p tetrahedron those matrices are built from, by definition:

Reference element  T = {xi >= 0, xi_1 + xi_2 + xi_3 <= 1}, barycentric coordinates
                   lambda = (1 - xi_1 - xi_2 - xi_3, xi_1, xi_2, xi_3).
Nodes              equispaced: multi-index (i, j, k), i + j + k <= p, at xi = (i, j, k) / p,
                   ordered k slowest, i fastest (the order of synthetic.simplex_multi_indices).
Basis              the equispaced Lagrange basis of P_p in Silvester's product form (P. Silvester,
                   "High-order polynomial triangular finite elements for potential problems",
                   Int. J. Eng. Sci. 7, 1969): with alpha = (p - i - j - k, i, j, k),
                       phi_alpha = prod_m R_{alpha_m}(lambda_m),
                       R_a(t) = prod_{s=0}^{a-1} (p t - s) / (s + 1),
                   which is 1 at its own node and 0 at every other node of the lattice.
Quadrature         conical product rule (Stroud, "Approximate calculation of multiple integrals",
                   1971): collapse xi = (u, (1-u) v, (1-u)(1-v) w), dV = (1-u)^2 (1-v) du dv dw on
                   [0,1]^3, Gauss-Jacobi in u (weight (1-u)^2) and v (weight (1-v)) and
                   Gauss-Legendre in w, q points each (nodes from scipy.special.roots_jacobi);
                   exact for polynomials of total degree <= 2q - 1.  Point order: the u index
                   fastest, then v, then w.
Geometry           affine: x(xi) = v0 + J xi with J = [v1 - v0, v2 - v0, v3 - v0] (columns).

The space object exposes the same attributes as fem.Space (Phi, dPhi, W, XI, nd, nq), so the
dense element action, assembly, Jacobi diagonal and PCG of fem apply unchanged.
"""
from __future__ import annotations

import numpy as np
from scipy.special import roots_jacobi

from . import fem


def multi_indices(p: int) -> np.ndarray:
    """(i, j, k) with i + j + k <= p, k slowest, i fastest."""
    return np.array([(i, j, k) for k in range(p + 1) for j in range(p + 1 - k) for i in range(p + 1 - j - k)],
                    dtype=np.int64)


def n_nodes(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def silvester_factor(a: int, p: int, t):
    """R_a(t) = prod_{s<a} (p t - s)/(s+1) and its derivative dR_a/dt (product rule, term by term)."""
    t = np.asarray(t, dtype=np.float64)
    R = np.ones_like(t)
    for s in range(a):
        R = R * (p * t - s) / (s + 1)
    dR = np.zeros_like(t)
    for s in range(a):
        term = np.full_like(t, p / (s + 1))
        for s2 in range(a):
            if s2 != s:
                term = term * (p * t - s2) / (s2 + 1)
        dR = dR + term
    return R, dR


def basis(p: int, xi):
    """Phi [npts, nd] and reference gradients dPhi [3, npts, nd] of the degree-p basis at xi [npts, 3]."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    lam = np.stack([1.0 - xi.sum(1), xi[:, 0], xi[:, 1], xi[:, 2]], 0)     # [4, npts]
    mi = multi_indices(p)
    nd = mi.shape[0]
    Phi = np.empty((xi.shape[0], nd))
    dPhi = np.empty((3, xi.shape[0], nd))
    for n, (i, j, k) in enumerate(mi):
        alpha = (p - i - j - k, i, j, k)
        R, dR = zip(*(silvester_factor(alpha[m], p, lam[m]) for m in range(4)))
        Phi[:, n] = R[0] * R[1] * R[2] * R[3]
        # d phi / d lambda_m, then d lambda_0 / d xi_d = -1 and d lambda_{d+1} / d xi_d = 1
        dl = [dR[m] * np.prod([R[o] for o in range(4) if o != m], axis=0) for m in range(4)]
        for d in range(3):
            dPhi[d, :, n] = dl[d + 1] - dl[0]
    return Phi, dPhi


def nodes(p: int) -> np.ndarray:
    """Reference coordinates [nd, 3] of the equispaced nodes."""
    return multi_indices(p).astype(np.float64) / p


def gauss_jacobi01(q: int, alpha: int):
    """q-point Gauss rule on [0, 1] for the weight (1 - u)^alpha."""
    t, w = roots_jacobi(q, alpha, 0)
    return (1.0 + t) / 2.0, w / 2.0 ** (alpha + 1)


def conical_rule(q: int):
    """Points XI [q^3, 3] and weights W [q^3] of the collapsed (conical product) rule on T."""
    u, wu = gauss_jacobi01(q, 2)
    v, wv = gauss_jacobi01(q, 1)
    w, ww = gauss_jacobi01(q, 0)
    # point index a + q (b + q c): u_a fastest, then v_b, then w_c
    idx = np.arange(q ** 3)
    iu, iv, iw = idx % q, (idx // q) % q, idx // (q * q)
    U, V, Wc = u[iu], v[iv], w[iw]
    XI = np.stack([U, (1.0 - U) * V, (1.0 - U) * (1.0 - V) * Wc], -1)
    W = wu[iu] * wv[iv] * ww[iw]
    return XI, W


class SimplexSpace:
    """Degree-p tetrahedron with the conical rule of q points per collapsed direction."""

    def __init__(self, p: int, q: int | None = None):
        if p < 1:
            raise ValueError("p >= 1")
        self.p = p
        self.q = p + 1 if q is None else q
        self.XI, self.W = conical_rule(self.q)
        self.Phi, self.dPhi = basis(p, self.XI)
        self.nd, self.nq = self.Phi.shape[1], self.Phi.shape[0]
        self.node_xi = nodes(p)


def affine_map(vertices, XI):
    """Physical points X [E, nq, 3] and the constant Jacobian J [E, 3, 3], J[:, a, b] = dx_a/dxi_b."""
    V = np.asarray(vertices, dtype=np.float64)
    J = np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]], -1)
    X = V[:, None, 0, :] + np.einsum("eab,qb->eqa", J, XI)
    return X, J


def qdata_mass(space: SimplexSpace, vertices, rho=None):
    """w_q |det J| rho_q, [E, nq]."""
    _, J = affine_map(vertices, space.XI)
    qd = space.W[None, :] * np.abs(np.linalg.det(J))[:, None]
    return qd if rho is None else qd * rho


def qdata_diffusion(space: SimplexSpace, vertices, k=None):
    """G_q = k_q w_q |det J| J^{-1} J^{-T}, [E, nq, 3, 3]; k None (1), 'sine' or [E, nq]."""
    X, J = affine_map(vertices, space.XI)
    Ji = np.linalg.inv(J)
    G = (space.W[None, :, None, None] * np.abs(np.linalg.det(J))[:, None, None, None]
         * (Ji @ np.swapaxes(Ji, -1, -2))[:, None, :, :])
    if k is None:
        return G
    if isinstance(k, str):
        if k != "sine":
            raise ValueError(k)
        k = fem.coeff_sine(X)
    return np.asarray(k)[..., None, None] * G


def node_points(p: int, vertices) -> np.ndarray:
    """Physical positions [E, nd, 3] of every element's nodes."""
    X, _ = affine_map(vertices, nodes(p))
    return X


def manufactured_rhs(space: SimplexSpace, vertices, elem_dofs, n: int, coeff: str = "sine", mask=None):
    """b_i = sum_e sum_q w_q |det J| f(x_q) phi_i(x_q) for u* = sin(pi x) sin(pi y) sin(pi z)."""
    X, J = affine_map(vertices, space.XI)
    fq = space.W[None, :] * np.abs(np.linalg.det(J))[:, None] * fem.manufactured_source(X, coeff)
    be = np.einsum("qn,eq->en", space.Phi, fq)
    b = np.zeros(n)
    np.add.at(b, elem_dofs.reshape(-1), be.reshape(-1))
    if mask is not None:
        b[np.asarray(mask).astype(bool)] = 0.0
    return b


def l2_error(p: int, vertices, elem_dofs, u, qextra: int = 3):
    """||u_h - u*||_{L2} with the conical rule of p + qextra points per direction."""
    sp_ = SimplexSpace(p, p + qextra)
    X, J = affine_map(vertices, sp_.XI)
    uh = np.einsum("qn,en->eq", sp_.Phi, u[elem_dofs])
    err = (uh - fem.exact_solution(X)) ** 2
    return float(np.sqrt(np.sum(sp_.W[None, :] * np.abs(np.linalg.det(J))[:, None] * err)))


def cost_model(space: SimplexSpace, op: str):
    """Per-element flops of the dense (GEMM) formulation: 2 nq nd multiply-adds per basis matrix and
    direction, forward and transposed (mass: 1 direction, diffusion: 3), plus the pointwise D."""
    dirs = 1 if op == fem.MASS else 3
    return 2 * 2 * dirs * space.nq * space.nd + (1 if op == fem.MASS else 15) * space.nq

"""Overlapping Schwarz smoother with fast diagonalization, for the oracle.  TEST INFRASTRUCTURE ONLY.

The paper lists Schwarz (fast diagonalization) smoothing beside p-multigrid and Chebyshev-Jacobi
as the preconditioners built on the same sum-factorized kernels (Section 1).  The method followed
is the overlapping Schwarz smoother of Lottes and Fischer ("Hybrid multigrid/Schwarz algorithms for
the spectral element method", J. Sci. Comput. 24, 2005), written out by definition:

  * each element's local problem lives on the element's own (p+1)^3 GLL nodes, with homogeneous
    Dirichlet conditions one node into each neighbouring element (the minimal overlap);
  * its operator is replaced by the separable one of a box of the element's mean side lengths
    (h_x, h_y, h_z) and mean coefficient k_e:
        A_e = k_e (B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x),
    with A_d = (2/h_d) A^, B_d = (h_d/2) B^ and (A^, B^) the 1D GLL stiffness and (diagonal) mass
    matrices of three reference elements assembled side by side, restricted to the middle element's
    nodes (the outer neighbours' next nodes are the Dirichlet nodes of the extension);
  * A_e is inverted exactly by fast diagonalization: A^ S = B^ S L, S^T B^ S = I, so
        A_e^{-1} = k_e^{-1} (2/h_x)(2/h_y)(2/h_z) (S (x) S (x) S) [4 L_x/h_x^2 + 4 L_y/h_y^2 + 4 L_z/h_z^2]^{-1}
                   (S (x) S (x) S)^T;
  * the element solutions are added with symmetric weights: z = sum_e R_e^T W A_e^{-1} W R_e r,
    W = diag(multiplicity^{-1/2}) (multiplicity: elements sharing the node); Dirichlet nodes are
    zero in r and z.
Mean side length h_d: the mean of the four element edges along reference axis d; k_e: the mean of
the coefficient over the element's GLL nodes (collocated quadrature points).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh

from . import fem
from .quadrature import gll, lagrange


def reference_1d(p: int):
    """(A^, B^) [p+1, p+1]: three reference elements assembled, restricted to the middle one."""
    x, w = gll(p + 1)
    _, dL = lagrange(x, x)                         # dL[q, j] = l_j'(x_q)
    K = np.einsum("q,qi,qj->ij", w, dL, dL)        # element stiffness on [-1, 1]
    n3 = 3 * p + 1
    A3, B3 = np.zeros((n3, n3)), np.zeros(n3)
    for el in range(3):
        s = el * p
        A3[s:s + p + 1, s:s + p + 1] += K
        B3[s:s + p + 1] += w
    mid = slice(p, 2 * p + 1)
    return A3[mid, mid], np.diag(B3[mid])


def fdm_1d(p: int):
    """(S, lam): A^ S = B^ S diag(lam), S^T B^ S = I."""
    A, B = reference_1d(p)
    lam, S = eigh(A, B)
    return S, lam


def element_lengths(vertices):
    """Mean side lengths [E, 3] of trilinear hexahedra (vertex v = vx + 2 vy + 4 vz)."""
    V = np.asarray(vertices, dtype=np.float64)
    h = np.zeros((V.shape[0], 3))
    for d in range(3):
        pairs = [(v, v | (1 << d)) for v in range(8) if not (v >> d) & 1]
        h[:, d] = np.mean([np.linalg.norm(V[:, b] - V[:, a], axis=-1) for a, b in pairs], axis=0)
    return h


def element_coefficient(p: int, vertices, coeff="sine"):
    """Mean coefficient over each element's GLL nodes [E] (1 for coeff None)."""
    if coeff is None:
        return np.ones(len(vertices))
    X = fem.node_points(p, vertices)
    return fem.coeff_sine(X).mean(axis=1)


def local_operator(p: int, h, k):
    """The separable element operator A_e [(p+1)^3]^2 (a fastest) for side lengths h and coefficient k."""
    A, B = reference_1d(p)
    Ad = [2.0 / h[d] * A for d in range(3)]
    Bd = [h[d] / 2.0 * B for d in range(3)]
    return k * (np.kron(Bd[2], np.kron(Bd[1], Ad[0])) + np.kron(Bd[2], np.kron(Ad[1], Bd[0]))
                + np.kron(Ad[2], np.kron(Bd[1], Bd[0])))


def local_solve(p: int, h, k, r):
    """A_e^{-1} r by fast diagonalization, r [(p+1)^3] with a fastest."""
    S, lam = fdm_1d(p)
    P = p + 1
    R = r.reshape(P, P, P)                         # [c, b, a]
    T = np.einsum("ai,cba->cbi", S, R)
    T = np.einsum("bj,cbi->cji", S, T)
    T = np.einsum("ck,cji->kji", S, T)
    lx, ly, lz = (4.0 / h[d] ** 2 * lam for d in range(3))
    T = T / (k * (lz[:, None, None] + ly[None, :, None] + lx[None, None, :]))
    T = np.einsum("ck,kji->cji", S, T)
    T = np.einsum("bj,cji->cbi", S, T)
    T = np.einsum("ai,cbi->cba", S, T)
    return T.reshape(-1) * (2.0 / h[0]) * (2.0 / h[1]) * (2.0 / h[2])


def schwarz(p: int, vertices, elem_dofs, n: int, mask=None, coeff="sine"):
    """Closure z = M r of the additive Schwarz smoother on an order-p mesh."""
    h = element_lengths(vertices)
    k = element_coefficient(p, vertices, coeff)
    mult = np.bincount(np.asarray(elem_dofs).reshape(-1), minlength=n).astype(np.float64)
    w = 1.0 / np.sqrt(mult)
    m = None if mask is None else np.asarray(mask).astype(bool)

    def apply(r):
        r = np.asarray(r, dtype=np.float64)
        if m is not None:
            r = np.where(m, 0.0, r)
        z = np.zeros(n)
        for e in range(len(elem_dofs)):
            idx = elem_dofs[e]
            z_e = local_solve(p, h[e], k[e], w[idx] * r[idx])
            np.add.at(z, idx, w[idx] * z_e)
        if m is not None:
            z[m] = 0.0
        return z
    return apply

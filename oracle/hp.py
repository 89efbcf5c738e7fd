"""Conforming hp (variable order) hexahedral spaces for the oracle.  TEST INFRASTRUCTURE ONLY.

The paper's mixed-order workload (elements of orders 3, 5, 7 in one launch) and its next step,
conforming hp interfaces, need a continuous finite-element space on a mesh whose elements have
different polynomial orders.  The reading taken here is the minimum rule: on a structured
nx*ny*nz hexahedral lattice (element e = ex + nx (ey + ny ez), order orders[e]), every face and
edge carries the lowest order of the elements that share it, and the space is

    V_h = { u continuous,  u|_e in Q_{p_e},  u restricted to a face/edge in Q_{p_entity} }.

It is the image of a conforming prolongation P from true degrees of freedom to element nodes
(each element's own GLL nodes, a + p+1 (b + (p+1) c)):
  * vertices carry one value each;
  * an edge of order p_E carries its interior GLL(p_E) nodes; the edge polynomial is the 1D
    Lagrange interpolant through its two vertices and those nodes;
  * a face of order p_F carries its interior GLL(p_F) x GLL(p_F) nodes; on its boundary the face
    polynomial takes the values of its edges' polynomials (which may have lower order still);
  * an element carries its interior nodes.
An element node is the value of the polynomial of the lowest-dimensional entity it lies on,
evaluated at the node; when the entity has the element's order the node is one of the entity's
own nodes and P has a single 1 in that row.  The operator on true dofs is P^T blockdiag(A_e) P
with A_e the dense element matrices of fem (Section 2's A^e for each element order).

Canonical true-dof numbering (shared with the C-ABI's hp handle):
  1. vertices (i, j, k), i fastest, (nx+1)(ny+1)(nz+1) of them;
  2. edges along x, then y, then z; within an axis by lower vertex (i, j, k), i fastest; each
     edge's interior nodes in increasing coordinate;
  3. faces normal to x, then y, then z; within an axis by lower corner (i, j, k), i fastest; each
     face's interior nodes with the first in-plane axis (the lower of the two other axes) fastest;
  4. element interiors in element order, a fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .quadrature import gll, lagrange

_RULES = {}


def _gll(p):
    if p not in _RULES:
        _RULES[p] = gll(p + 1)[0]
    return _RULES[p]


def _weights(p, t):
    """Lagrange weights of the GLL(p) nodes at the point t (exact 0/1 at the nodes themselves)."""
    L, _ = lagrange(_gll(p), [t])
    return L[0]


class HpSpace:
    """Conforming variable-order space on an nx*ny*nz lattice (see the module docstring)."""

    def __init__(self, nx, ny, nz, orders):
        self.n = (nx, ny, nz)
        self.orders = np.asarray(orders, dtype=np.int64).reshape(-1)
        if self.orders.size != nx * ny * nz or self.orders.min() < 1:
            raise ValueError("one order >= 1 per element")
        self._entity_orders()
        self._number()
        self._prolongation()

    # ------------------------------------------------------------------ entities
    def elem_order(self, ex, ey, ez):
        nx, ny, _ = self.n
        return int(self.orders[ex + nx * (ey + ny * ez)])

    def _entity_orders(self):
        nx, ny, nz = self.n
        big = 1 << 30
        # edge along axis d at lower vertex v: shared by the elements with that lattice edge
        self.edge_order = {}
        self.face_order = {}
        for d in range(3):
            ext = [nx + 1, ny + 1, nz + 1]
            ext[d] -= 1
            for k in range(ext[2]):
                for j in range(ext[1]):
                    for i in range(ext[0]):
                        v = [i, j, k]
                        o = [a for a in range(3) if a != d]
                        best = big
                        for s0 in (-1, 0):
                            for s1 in (-1, 0):
                                c = list(v)
                                c[o[0]] += s0
                                c[o[1]] += s1
                                if 0 <= c[0] < nx and 0 <= c[1] < ny and 0 <= c[2] < nz:
                                    best = min(best, self.elem_order(*c))
                        self.edge_order[(d, i, j, k)] = best
            fext = [nx, ny, nz]
            fext[d] += 1
            for k in range(fext[2]):
                for j in range(fext[1]):
                    for i in range(fext[0]):
                        v = [i, j, k]
                        best = big
                        for s in (-1, 0):
                            c = list(v)
                            c[d] += s
                            if 0 <= c[0] < nx and 0 <= c[1] < ny and 0 <= c[2] < nz:
                                best = min(best, self.elem_order(*c))
                        self.face_order[(d, i, j, k)] = best

    def _number(self):
        nx, ny, nz = self.n
        nid = 0
        self.vertex_dof = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
        nid = (nx + 1) * (ny + 1) * (nz + 1)
        self.edge_dof = {}
        for d in range(3):
            keys = sorted((key for key in self.edge_order if key[0] == d), key=lambda t: (t[3], t[2], t[1]))
            for key in keys:
                p = self.edge_order[key]
                for m in range(1, p):
                    self.edge_dof[key + (m,)] = nid
                    nid += 1
        self.face_dof = {}
        for d in range(3):
            keys = sorted((key for key in self.face_order if key[0] == d), key=lambda t: (t[3], t[2], t[1]))
            for key in keys:
                p = self.face_order[key]
                for m2 in range(1, p):
                    for m1 in range(1, p):
                        self.face_dof[key + (m1, m2)] = nid
                        nid += 1
        self.cell_dof0 = np.zeros(nx * ny * nz, dtype=np.int64)
        for e in range(nx * ny * nz):
            self.cell_dof0[e] = nid
            nid += (int(self.orders[e]) - 1) ** 3
        self.n_true = nid

    # ------------------------------------------------------------------ entity polynomials
    def value_at_edge(self, key, t):
        """Row {true dof: weight} of the edge polynomial at reference coordinate t in [-1, 1]."""
        d, i, j, k = key
        p = self.edge_order[key]
        w = _weights(p, t)
        row = {}
        lo = [i, j, k]
        hi = list(lo)
        hi[d] += 1
        for m in range(p + 1):
            if w[m] == 0.0:
                continue
            if m == 0:
                dofs = {self.vertex_dof(*lo): 1.0}
            elif m == p:
                dofs = {self.vertex_dof(*hi): 1.0}
            else:
                dofs = {self.edge_dof[key + (m,)]: 1.0}
            for q, c in dofs.items():
                row[q] = row.get(q, 0.0) + w[m] * c
        return row

    def value_at_face(self, key, s, t):
        """Row of the face polynomial at in-plane reference coordinates (s, t) (first, second axis)."""
        d, i, j, k = key
        o0, o1 = [a for a in range(3) if a != d]
        p = self.face_order[key]
        xs = _gll(p)
        ws, wt = _weights(p, s), _weights(p, t)
        row = {}
        for m1 in range(p + 1):
            if ws[m1] == 0.0:
                continue
            for m2 in range(p + 1):
                if wt[m2] == 0.0:
                    continue
                b1, b2 = m1 in (0, p), m2 in (0, p)
                corner = [i, j, k]
                if b1 and b2:
                    corner[o0] += 1 if m1 == p else 0
                    corner[o1] += 1 if m2 == p else 0
                    sub = {self.vertex_dof(*corner): 1.0}
                elif b1:    # on the face's edge along the second in-plane axis
                    corner[o0] += 1 if m1 == p else 0
                    sub = self.value_at_edge((o1, *corner), xs[m2])
                elif b2:    # on the edge along the first in-plane axis
                    corner[o1] += 1 if m2 == p else 0
                    sub = self.value_at_edge((o0, *corner), xs[m1])
                else:
                    sub = {self.face_dof[key + (m1, m2)]: 1.0}
                wgt = ws[m1] * wt[m2]
                for q, c in sub.items():
                    row[q] = row.get(q, 0.0) + wgt * c
        return row

    def node_row(self, e, a, b, c):
        """Row of P for node (a, b, c) of element e."""
        nx, ny, _ = self.n
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        p = int(self.orders[e])
        x = _gll(p)
        idx = (a, b, c)
        base = (ex, ey, ez)
        bnd = [t in (0, p) for t in idx]
        nb = sum(bnd)
        if nb == 3:
            v = [base[d] + (1 if idx[d] == p else 0) for d in range(3)]
            return {self.vertex_dof(*v): 1.0}
        if nb == 2:
            d = bnd.index(False)
            v = [base[a_] + (1 if (a_ != d and idx[a_] == p) else 0) for a_ in range(3)]
            return self.value_at_edge((d, *v), x[idx[d]])
        if nb == 1:
            d = bnd.index(True)
            v = list(base)
            v[d] += 1 if idx[d] == p else 0
            o0, o1 = [a_ for a_ in range(3) if a_ != d]
            return self.value_at_face((d, *v), x[idx[o0]], x[idx[o1]])
        P = p - 1
        return {int(self.cell_dof0[e]) + (a - 1) + P * ((b - 1) + P * (c - 1)): 1.0}

    def _prolongation(self):
        """P [sum_e (p_e+1)^3, n_true] (CSR), rows in element order, element nodes a fastest."""
        rows, cols, vals = [], [], []
        self.row0 = np.zeros(len(self.orders) + 1, dtype=np.int64)
        r = 0
        for e, p in enumerate(self.orders):
            self.row0[e] = r
            P = int(p) + 1
            for c in range(P):
                for b in range(P):
                    for a in range(P):
                        for q, w in self.node_row(e, a, b, c).items():
                            rows.append(r)
                            cols.append(q)
                            vals.append(w)
                        r += 1
        self.row0[-1] = r
        self.P = sp.csr_matrix((vals, (rows, cols)), shape=(r, self.n_true))

    # ------------------------------------------------------------------ geometry helpers
    def boundary_mask(self):
        """True dofs on the boundary of the lattice (Dirichlet nodes)."""
        nx, ny, nz = self.n
        m = np.zeros(self.n_true, dtype=bool)
        for k in range(nz + 1):
            for j in range(ny + 1):
                for i in range(nx + 1):
                    if i in (0, nx) or j in (0, ny) or k in (0, nz):
                        m[self.vertex_dof(i, j, k)] = True
        lim = (nx, ny, nz)
        for (d, i, j, k, *_), q in self.edge_dof.items():
            v = (i, j, k)
            if any(v[a] in (0, lim[a]) for a in range(3) if a != d):
                m[q] = True
        for (d, i, j, k, *_), q in self.face_dof.items():
            if (i, j, k)[d] in (0, lim[d]):
                m[q] = True
        return m


def element_spaces(hp: HpSpace, qkind: str):
    return {int(p): fem.Space(int(p), qkind) for p in np.unique(hp.orders)}


def operator(hp: HpSpace, vertices, qkind: str, op: str, coeff="sine"):
    """Closure y = P^T blockdiag(A_e) P x on true dofs (dense element actions, element order)."""
    spaces = element_spaces(hp, qkind)
    qd = {}
    for p, s_ in spaces.items():
        sel = np.nonzero(hp.orders == p)[0]
        if op == fem.DIFFUSION:
            qd[p] = (sel, fem.qdata_diffusion(s_, vertices[sel], coeff))
        else:
            rho = None
            if coeff == "sine":
                X, _ = fem.trilinear_map(vertices[sel], s_.XI)
                rho = fem.coeff_sine(X)
            qd[p] = (sel, fem.qdata_mass(s_, vertices[sel], rho))

    def apply(x):
        uE = hp.P @ x
        yE = np.zeros_like(uE)
        for p, (sel, q) in qd.items():
            nd = (p + 1) ** 3
            idx = hp.row0[sel][:, None] + np.arange(nd)[None, :]
            yE[idx] = fem.element_action(spaces[p], uE[idx], q, op)
        return hp.P.T @ yE
    return apply


def element_values(hp: HpSpace, x):
    """E-vector P x split per element: list of arrays [(p_e+1)^3]."""
    uE = hp.P @ x
    return [uE[hp.row0[e]:hp.row0[e + 1]] for e in range(len(hp.orders))]

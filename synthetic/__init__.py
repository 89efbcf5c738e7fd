"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds no arithmetic of the finite-element method: it only makes
meshes (vertex coordinates, the element-to-DOF map, the boundary mask) and
random vectors/fields.  Everything is generated on the host with a
counter-based SplitMix64 stream (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so x86 and Arm hosts produce
bit-identical inputs.

Workload shapes follow the bake-off problems the paper benchmarks (Section 1,
BP1/BP3/BP5): a structured N^3 (or nx*ny*nz) hexahedral lattice of the unit
cube whose strictly interior vertices are moved by an independent uniform
offset in [-0.1h, 0.1h] per coordinate, Q_p elements with (p+1)^3 nodes,
nodes numbered lexicographically with x fastest.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags keep the different random quantities independent for one seed
TAG_VERTEX = 1
TAG_VECTOR = 2
TAG_FIELD = 3
TAG_DIRECTION = 4


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_seed(seed: int, tag: int) -> np.uint64:
    """Derive the starting state of an independent stream from (seed, tag)."""
    with np.errstate(over="ignore"):
        s = np.array([np.uint64(seed) ^ (np.uint64(tag) * _GOLDEN)], dtype=np.uint64)
        return _mix(s)[0]


def splitmix64(state0: np.uint64, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 begun at state0 (counter form)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(state0) + k * _GOLDEN)


def uniform01(bits: np.ndarray) -> np.ndarray:
    """Top 53 bits of each word as a double in [0, 1)."""
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, tag: int = TAG_VECTOR,
            chunk: int = 1 << 24) -> np.ndarray:
    """n doubles uniform in [lo, hi), generated in chunks to bound host memory."""
    out = np.empty(n, dtype=np.float64)
    s0 = stream_seed(seed, tag)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = lo + (hi - lo) * uniform01(splitmix64(s0, a, b - a))
    return out


def standard_normal(n: int, seed: int, tag: int = TAG_FIELD) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform on pairs of uniforms."""
    m = (n + 1) // 2
    s0 = stream_seed(seed, tag)
    u = uniform01(splitmix64(s0, 0, 2 * m))
    u1 = 1.0 - u[0::2]          # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def lognormal(n: int, seed: int, sigma: float = 0.5, tag: int = TAG_FIELD) -> np.ndarray:
    """exp(sigma z), z ~ N(0, 1): a positive coefficient with median 1."""
    return np.exp(sigma * standard_normal(n, seed, tag))


class HexMesh:
    """A structured nx*ny*nz hexahedral mesh of the unit cube with Q_p numbering.

    Attributes (all host numpy arrays):
      vertices  [E, 8, 3] float64, local vertex v = vx + 2 vy + 4 vz
      elem_dofs [E, (p+1)^3] int32, local node a + P (b + P c) (a fastest)
      boundary  [n_ldof] uint8, 1 on the boundary of the node lattice
    Element e = ex + nx (ey + ny ez); global node I + Mx (J + My K) with
    Mx = p nx + 1.
    """

    def __init__(self, nx: int, ny: int, nz: int, p: int, seed: int = 0, perturb: float = 0.1,
                 build_map: bool = True):
        if p < 1 or min(nx, ny, nz) < 1:
            raise ValueError("need p >= 1 and at least one element per direction")
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.P = p + 1
        self.n_elem = nx * ny * nz
        self.Mx, self.My, self.Mz = p * nx + 1, p * ny + 1, p * nz + 1
        self.n_ldof = self.Mx * self.My * self.Mz
        self.seed, self.perturb = seed, perturb
        self.vertex_lattice = self._vertex_lattice()
        self.vertices = self._element_vertices()
        self.elem_dofs = self._elem_dofs() if build_map else None
        self._boundary = None

    @property
    def boundary(self) -> np.ndarray:
        if self._boundary is None:
            I = np.arange(self.Mx)
            J = np.arange(self.My)
            K = np.arange(self.Mz)
            bI = (I == 0) | (I == self.Mx - 1)
            bJ = (J == 0) | (J == self.My - 1)
            bK = (K == 0) | (K == self.Mz - 1)
            b = bK[:, None, None] | bJ[None, :, None] | bI[None, None, :]
            self._boundary = b.reshape(-1).astype(np.uint8)
        return self._boundary

    def _vertex_lattice(self) -> np.ndarray:
        nx, ny, nz = self.nx, self.ny, self.nz
        gx = np.arange(nx + 1) / nx
        gy = np.arange(ny + 1) / ny
        gz = np.arange(nz + 1) / nz
        X = np.empty((nz + 1, ny + 1, nx + 1, 3))
        X[..., 0] = gx[None, None, :]
        X[..., 1] = gy[None, :, None]
        X[..., 2] = gz[:, None, None]
        if self.perturb > 0:
            n = X.shape[0] * X.shape[1] * X.shape[2]
            u = uniform01(splitmix64(stream_seed(self.seed, TAG_VERTEX), 0, 3 * n)).reshape(X.shape)
            h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
            off = (2.0 * u - 1.0) * self.perturb * h
            inner = np.zeros(X.shape[:3], dtype=bool)
            inner[1:nz, 1:ny, 1:nx] = True
            X[inner] += off[inner]
        return X

    def _element_vertices(self) -> np.ndarray:
        nx, ny, nz = self.nx, self.ny, self.nz
        X = self.vertex_lattice
        V = np.empty((nz, ny, nx, 8, 3))
        for v in range(8):
            vx, vy, vz = v & 1, (v >> 1) & 1, (v >> 2) & 1
            V[:, :, :, v, :] = X[vz:vz + nz, vy:vy + ny, vx:vx + nx, :]
        return V.reshape(self.n_elem, 8, 3)

    def _elem_dofs(self) -> np.ndarray:
        p, P = self.p, self.P
        nx, ny, nz = self.nx, self.ny, self.nz
        a = np.arange(P)
        base = (p * np.arange(nx))[None, None, :] + self.Mx * (
            (p * np.arange(ny))[None, :, None] + self.My * (p * np.arange(nz))[:, None, None])
        local = a[None, None, :] + self.Mx * (a[None, :, None] + self.My * a[:, None, None])
        dofs = base.reshape(-1, 1) + local.reshape(1, -1)
        if self.n_ldof >= 2 ** 31:
            raise ValueError("node count exceeds int32 indexing")
        return dofs.astype(np.int32)

    def interior_dof_count(self) -> int:
        """Nodes off the boundary: (p nx - 1)(p ny - 1)(p nz - 1)."""
        return (self.Mx - 2) * (self.My - 2) * (self.Mz - 2)


def bubble_warp(X: np.ndarray, amplitude: float = 0.05) -> np.ndarray:
    """A smooth deformation of the unit cube that keeps its boundary fixed (curved-mesh inputs).

    x -> x + amplitude * b(x) * (1, -0.75, 0.5) with the bubble b = 64 x(1-x) y(1-y) z(1-z)
    (zero on every face, 1 at the centre).  |grad b| <= 4 per component, so the map stays
    invertible for amplitude < 1/9.  X [..., 3] physical points; returns the moved points.
    """
    X = np.asarray(X, dtype=np.float64)
    b = 64.0 * np.prod(X * (1.0 - X), axis=-1)
    return X + amplitude * b[..., None] * np.array([1.0, -0.75, 0.5])


def cube_mesh(N: int, p: int, seed: int = 0, perturb: float = 0.1, build_map: bool = True) -> HexMesh:
    return HexMesh(N, N, N, p, seed=seed, perturb=perturb, build_map=build_map)


# Kuhn (Freudenthal) split of a cube into 6 tetrahedra: one per ordering of the axes, the path
# 0 -> e_s0 -> e_s0 + e_s1 -> (1, 1, 1).  Listed with the sign of the permutation.
KUHN_PATHS = (((0, 1, 2), 1), ((0, 2, 1), -1), ((1, 0, 2), -1), ((1, 2, 0), 1), ((2, 0, 1), 1), ((2, 1, 0), -1))


def simplex_multi_indices(p: int) -> np.ndarray:
    """Local node order of a degree-p tetrahedron: multi-indices (i, j, k), i + j + k <= p, with
    k slowest and i fastest; node (i, j, k) sits at xi = (i, j, k) / p of the reference element."""
    out = [(i, j, k) for k in range(p + 1) for j in range(p + 1 - k) for i in range(p + 1 - j - k)]
    return np.array(out, dtype=np.int64)


class TetMesh:
    """Tetrahedral mesh of the unit cube: every cube of the perturbed nx*ny*nz lattice (the same
    vertex positions as HexMesh) split into the 6 Kuhn tetrahedra, with degree-p nodes.

    Attributes (host numpy arrays):
      vertices  [E, 4, 3] float64: the element's vertices v0..v3; the element map is
                x(xi) = v0 + sum_d xi_d (v_{d+1} - v0) on the reference tetrahedron
                {xi >= 0, xi_1 + xi_2 + xi_3 <= 1}
      elem_dofs [E, (p+1)(p+2)(p+3)/6] int32 in the order of simplex_multi_indices(p)
      boundary  [n_ldof] uint8
    Element e = 6 c + t for cube c = ex + nx (ey + ny ez) and path t of KUHN_PATHS; paths of odd
    permutations list their last two vertices swapped, so every element has a positive volume on
    the unperturbed lattice.  The equispaced degree-p nodes of every element are points of the
    lattice refined p times, so the global node of local node (i, j, k) is that lattice point:
    nodes shared by neighbouring elements get one number, and n_ldof = (p nx + 1)(p ny + 1)(p nz + 1).
    """

    def __init__(self, nx: int, ny: int, nz: int, p: int, seed: int = 0, perturb: float = 0.1):
        if p < 1 or min(nx, ny, nz) < 1:
            raise ValueError("need p >= 1 and at least one cube per direction")
        hexes = HexMesh(nx, ny, nz, p, seed=seed, perturb=perturb, build_map=False)
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.n_elem = 6 * nx * ny * nz
        self.Mx, self.My, self.Mz = hexes.Mx, hexes.My, hexes.Mz
        self.n_ldof = hexes.n_ldof
        self.boundary = hexes.boundary
        corners = np.zeros((6, 4, 3), dtype=np.int64)       # lattice offsets of v0..v3 per path
        for t, (perm, sign) in enumerate(KUHN_PATHS):
            c = [np.zeros(3, np.int64)]
            for a in perm:
                c.append(c[-1].copy())
                c[-1][a] += 1
            if sign < 0:
                c[2], c[3] = c[3], c[2]
            corners[t] = np.array(c)
        self.corners = corners
        X = hexes.vertex_lattice                              # [nz+1, ny+1, nx+1, 3]
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
        V = np.empty((nx * ny * nz, 6, 4, 3))
        for t in range(6):
            for v in range(4):
                cx, cy, cz = corners[t, v]
                V[:, t, v, :] = X[ez + cz, ey + cy, ex + cx]
        self.vertices = V.reshape(self.n_elem, 4, 3)
        mi = simplex_multi_indices(p)                         # [nd, 3]
        # lattice offset of node (i, j, k): i c1 + j c2 + k c3 (c0 is the cube's origin corner)
        off = np.einsum("nk,tkc->tnc", mi, corners[:, 1:, :])  # [6, nd, 3]
        base = np.stack([p * ex, p * ey, p * ez], -1)          # [cubes, 3]
        L = base[:, None, None, :] + off[None, :, :, :]        # [cubes, 6, nd, 3]
        dofs = L[..., 0] + self.Mx * (L[..., 1] + self.My * L[..., 2])
        self.elem_dofs = dofs.reshape(self.n_elem, -1).astype(np.int32)
        self.nd = mi.shape[0]


def tet_cube_mesh(N: int, p: int, seed: int = 0, perturb: float = 0.1) -> TetMesh:
    return TetMesh(N, N, N, p, seed=seed, perturb=perturb)

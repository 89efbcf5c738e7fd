"""Thin Python binding of libceedgb.so (the GB300 matrix-free hexahedral operator library).

Every function here has the name of the C entry point it wraps (include/ceed_gb300.h) and only
marshals arguments: torch CUDA tensors become device pointers, the current torch stream becomes
the cudaStream_t.  All work runs in the library's CUDA kernels; there is no fallback path, and
importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB

# ceed_status
CEED_OK, CEED_ERR_INVALID, CEED_ERR_CUDA, CEED_ERR_OOM = 0, 1, 2, 3
CEED_ERR_NOT_CONVERGED, CEED_ERR_UNSUPPORTED, CEED_ERR_BAD_GEOMETRY = 4, 5, 6
CEED_ERR_TIMEOUT, CEED_ERR_NONFINITE = 7, 8
# ceed_prec
CEED_F64, CEED_F32, CEED_BF16, CEED_F16, CEED_F32_GEO, CEED_F64_DF = 0, 1, 2, 3, 4, 5
# ceed_qrule / ceed_op / ceed_coeff
CEED_QRULE_GLL, CEED_QRULE_GAUSS = 0, 1
CEED_OP_MASS, CEED_OP_DIFFUSION = 0, 1
CEED_COEFF_ONE, CEED_COEFF_CONST, CEED_COEFF_SINE, CEED_COEFF_PER_QPT = 0, 1, 2, 3
CEED_APPLY_DIRICHLET = 1
CEED_APPLY_F64_DF = 2
CEED_CG_FP64, CEED_CG_MIXED, CEED_CG_MIXED_RELIABLE = 0, 1, 2
CEED_NT_FUSED, CEED_NT_GEMM, CEED_NT_TC = 0, 1, 2

PREC_BYTES = {CEED_F64: 8, CEED_F32: 4, CEED_BF16: 2, CEED_F16: 2, CEED_F32_GEO: 4, CEED_F64_DF: 8}


class CeedError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ceed status {status}: {msg}")
        self.status = status


class _MeshDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_ldof", ctypes.c_int64), ("p", ctypes.c_int32),
                ("q_rule", ctypes.c_int32), ("n_qpts_1d", ctypes.c_int32), ("ncomp", ctypes.c_int32),
                ("elem_dofs", ctypes.c_void_p), ("vertices", ctypes.c_void_p), ("dirichlet", ctypes.c_void_p),
                ("coords", ctypes.c_void_p)]


class _CgOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("fixed_iters", ctypes.c_int32), ("op", ctypes.c_int32),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("qdata_lo", ctypes.c_void_p),
                ("prec_lo", ctypes.c_int32), ("use_x0", ctypes.c_int32), ("pmg", ctypes.c_void_p),
                ("reliable_delta", ctypes.c_double), ("separate_kernels", ctypes.c_int32)]


class _PmgOpts(ctypes.Structure):
    _fields_ = [("smooth_degree", ctypes.c_int32), ("smooth_ratio", ctypes.c_double), ("eig_iters", ctypes.c_int32),
                ("coarse_tol", ctypes.c_double), ("coarse_max_iter", ctypes.c_int32), ("prec_lo", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("smoother_coeff", ctypes.c_int32)]


class _NtDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_ldof", ctypes.c_int64), ("P", ctypes.c_int32), ("Q", ctypes.c_int32),
                ("interp", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("qweight", ctypes.c_void_p),
                ("qref", ctypes.c_void_p), ("elem_dofs", ctypes.c_void_p), ("vertices", ctypes.c_void_p),
                ("dirichlet", ctypes.c_void_p)]


class _HpDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("orders", ctypes.c_void_p),
                ("vertices", ctypes.c_void_p), ("q_rule", ctypes.c_int32), ("dirichlet", ctypes.c_int32)]


class _CgReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("fused", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"libceedgb.so is not built ({LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB)
    vp, i32, i64, u32, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ceed_setup_mesh": (ctypes.c_int, [ctypes.POINTER(_MeshDesc), ctypes.POINTER(vp), vp]),
        "ceed_destroy_mesh": (ctypes.c_int, [vp]),
        "ceed_mesh_node_coords": (ctypes.c_int, [vp, vp, vp]),
        "ceed_mesh_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ceed_mesh_bricks": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
        "ceed_qdata_bytes": (sz, [vp, ctypes.c_int, ctypes.c_int]),
        "ceed_build_qdata": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp]),
        "ceed_apply_mass": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, ctypes.c_int, u32, vp]),
        "ceed_apply_diffusion": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, ctypes.c_int, u32, vp]),
        "ceed_apply_host": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, u32,
                                           vp]),
        "ceed_jacobi_diagonal": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, u32, vp]),
        "ceed_schwarz_fdm_1d": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "ceed_hp_prolongation": (ctypes.c_int, [i32, i32, i32, vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                                ctypes.POINTER(i64), vp, vp, vp, vp]),
        "ceed_set_apply_variant": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "ceed_autotune_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_int,
                                               ctypes.POINTER(i32), ctypes.POINTER(i32),
                                               ctypes.POINTER(ctypes.c_float), vp]),
        "ceed_manufactured_rhs": (ctypes.c_int, [vp, ctypes.c_int, vp, u32, vp]),
        "ceed_cg_workspace_bytes": (sz, [vp, ctypes.POINTER(_CgOpts)]),
        "ceed_cg_solve": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, ctypes.POINTER(_CgOpts),
                                         ctypes.POINTER(_CgReport), vp, sz, vp]),
        "ceed_build_geometry": (ctypes.c_int, [vp, vp, vp]),
        "ceed_pmg_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(_PmgOpts), ctypes.POINTER(vp), vp]),
        "ceed_pmg_vcycle": (ctypes.c_int, [vp, vp, vp, vp]),
        "ceed_pmg_prolong": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp]),
        "ceed_pmg_restrict": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp]),
        "ceed_pmg_info": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "ceed_pmg_destroy": (ctypes.c_int, [vp]),
        "ceed_apply_diffusion_k": (ctypes.c_int, [vp, vp, vp, vp, vp, u32, vp]),
        "ceed_apply_diffusion_adjoint": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, u32, vp]),
        "ceed_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                             ctypes.POINTER(vp)]),
        "ceed_batch_apply": (ctypes.c_int, [vp, vp]),
        "ceed_batch_autotune": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), vp]),
        "ceed_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint32)]),
        "ceed_batch_status": (ctypes.c_int, [vp, vp]),
        "ceed_mesh_status": (ctypes.c_int, [vp, vp]),
        "ceed_set_wait_limits": (ctypes.c_int, [i64, i64]),
        "ceed_fma_throughput": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                               ctypes.POINTER(dbl), vp]),
        "ceed_batch_destroy": (ctypes.c_int, [vp]),
        "ceed_simplex_sizes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ceed_simplex_basis": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]),
        "ceed_nt_setup": (ctypes.c_int, [ctypes.POINTER(_NtDesc), ctypes.POINTER(vp), vp]),
        "ceed_nt_destroy": (ctypes.c_int, [vp]),
        "ceed_nt_qdata_bytes": (sz, [vp, ctypes.c_int, ctypes.c_int]),
        "ceed_nt_build_qdata": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp]),
        "ceed_nt_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, u32, vp]),
        "ceed_nt_set_algorithm": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int]),
        "ceed_nt_get_algorithm": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(i32),
                                                 ctypes.POINTER(i64), ctypes.POINTER(i32),
                                                 ctypes.POINTER(ctypes.c_float)]),
        "ceed_nt_autotune": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
        "ceed_nt_status": (ctypes.c_int, [vp, vp]),
        "ceed_schwarz_create": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.POINTER(vp), vp]),
        "ceed_schwarz_apply": (ctypes.c_int, [vp, vp, vp, u32, vp]),
        "ceed_schwarz_destroy": (ctypes.c_int, [vp]),
        "ceed_hp_setup": (ctypes.c_int, [ctypes.POINTER(_HpDesc), ctypes.POINTER(vp), vp]),
        "ceed_hp_destroy": (ctypes.c_int, [vp]),
        "ceed_hp_info": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        "ceed_hp_build_qdata": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp]),
        "ceed_hp_prolong": (ctypes.c_int, [vp, vp, vp, vp]),
        "ceed_hp_apply": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, u32, vp]),
        "ceed_dot_workspace_bytes": (sz, [i64]),
        "ceed_dot": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "ceed_dot_noalloc_max_n": (i64, []),
        "ceed_dot_noalloc": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "ceed_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib, sig


_lib, _SIGNATURES = _load()
EXPORTED = tuple(_SIGNATURES)


def _check(st):
    if st != CEED_OK:
        raise CeedError(st, _lib.ceed_last_error().decode())
    return st


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor (the library computes on the GPU only)")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    """Address of a contiguous FP64 host tensor (a host buffer of ceed_apply_host)."""
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64:
        raise ValueError("expected a contiguous float64 host tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Mesh:
    """Owns a ceed_mesh_t; the C handle is released on close() or garbage collection."""

    def __init__(self, handle, n_elem, n_ldof, p, q_rule, ncomp):
        self.handle = handle
        self.n_elem, self.n_ldof, self.p, self.q_rule, self.ncomp = n_elem, n_ldof, p, q_rule, ncomp
        nc, Q, P = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.ceed_mesh_info(handle, ctypes.byref(nc), ctypes.byref(Q), ctypes.byref(P)))
        self.n_colors, self.Q, self.P = nc.value, Q.value, P.value
        self.nq = self.Q ** 3

    def close(self):
        if self.handle:
            _lib.ceed_destroy_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_setup_mesh(n_elem, n_ldof, p, elem_dofs, vertices, dirichlet=None, q_rule=CEED_QRULE_GLL, n_qpts_1d=0,
                    ncomp=1, stream=None, coords=None) -> Mesh:
    assert elem_dofs.dtype == torch.int32 and vertices.dtype == torch.float64
    assert dirichlet is None or dirichlet.dtype == torch.uint8
    assert coords is None or (coords.dtype == torch.float64 and coords.is_contiguous())
    d = _MeshDesc(n_elem, n_ldof, p, q_rule, n_qpts_1d, ncomp, _ptr(elem_dofs), _ptr(vertices), _ptr(dirichlet),
                  _ptr(coords))
    h = ctypes.c_void_p()
    _check(_lib.ceed_setup_mesh(ctypes.byref(d), ctypes.byref(h), _stream(stream)))
    return Mesh(h, n_elem, n_ldof, p, q_rule, ncomp)


def ceed_mesh_info(mesh: Mesh):
    """(n_colors, Q, P) of a mesh handle."""
    nc, Q, P = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ceed_mesh_info(mesh.handle, ctypes.byref(nc), ctypes.byref(Q), ctypes.byref(P)))
    return nc.value, Q.value, P.value


def ceed_mesh_bricks(mesh: Mesh) -> int:
    """Number of 2 x 2 x 2 element bricks found at setup (0: the mesh is not a brick lattice)."""
    n = ctypes.c_int64()
    _check(_lib.ceed_mesh_bricks(mesh.handle, ctypes.byref(n)))
    return n.value


def ceed_mesh_node_coords(mesh: Mesh, coords: torch.Tensor, stream=None):
    """Physical node positions [n_ldof, 3] (curved copy, or the trilinear map at the GLL nodes)."""
    assert coords.dtype == torch.float64 and coords.is_contiguous() and coords.numel() == 3 * mesh.n_ldof
    _check(_lib.ceed_mesh_node_coords(mesh.handle, _ptr(coords), _stream(stream)))


def ceed_destroy_mesh(mesh: Mesh):
    mesh.close()


def ceed_qdata_bytes(mesh: Mesh, op: int, prec: int) -> int:
    return int(_lib.ceed_qdata_bytes(mesh.handle, op, prec))


def alloc_qdata(mesh: Mesh, op: int, prec: int, device=None) -> torch.Tensor:
    """Caller-owned quadrature-data buffer of the right size (uint8 bytes)."""
    return torch.empty(ceed_qdata_bytes(mesh, op, prec), dtype=torch.uint8, device=device or "cuda")


def ceed_build_qdata(mesh: Mesh, op, coeff_kind, coeff, prec, qdata, stream=None):
    if coeff_kind == CEED_COEFF_CONST:
        cval = (ctypes.c_double * 1)(float(coeff))
        cptr = ctypes.cast(cval, ctypes.c_void_p)
    else:
        cptr = _ptr(coeff) if coeff is not None else None
    _check(_lib.ceed_build_qdata(mesh.handle, op, coeff_kind, cptr, prec, _ptr(qdata), _stream(stream)))


def ceed_apply_mass(mesh: Mesh, qdata, prec, x, y, nrhs=1, flags=0, stream=None):
    _check(_lib.ceed_apply_mass(mesh.handle, _ptr(qdata), prec, _ptr(x), _ptr(y), nrhs, flags, _stream(stream)))


def ceed_apply_diffusion(mesh: Mesh, qdata, prec, x, y, nrhs=1, flags=0, stream=None):
    _check(_lib.ceed_apply_diffusion(mesh.handle, _ptr(qdata), prec, _ptr(x), _ptr(y), nrhs, flags, _stream(stream)))


def ceed_apply_host(mesh: Mesh, op, qdata, prec, x_host, y_host, x_dev, y_dev, nrhs=1, flags=0, stream=None):
    """y_host = A x_host through the device buffers x_dev, y_dev (copies and apply on `stream`; returns when
    y_host holds the result)."""
    n = mesh.n_ldof * mesh.ncomp * nrhs
    for t in (x_host, y_host, x_dev, y_dev):
        if t.numel() < n:
            raise ValueError("buffer smaller than n_ldof * ncomp * nrhs")
    _check(_lib.ceed_apply_host(mesh.handle, op, _ptr(qdata), prec, _host_ptr(x_host), _host_ptr(y_host), _ptr(x_dev),
                                _ptr(y_dev), nrhs, flags, _stream(stream)))


def ceed_autotune_apply(mesh: Mesh, op, qdata, prec, x, y, nrhs=1, stream=None):
    """Time the apply variants on these buffers and keep the fastest; returns (ne, stage, ms)."""
    ne, st, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(_lib.ceed_autotune_apply(mesh.handle, op, _ptr(qdata), prec, _ptr(x), _ptr(y), nrhs, ctypes.byref(ne),
                                    ctypes.byref(st), ctypes.byref(ms), _stream(stream)))
    return ne.value, st.value, ms.value


def ceed_set_apply_variant(mesh: Mesh, op, prec, ne, stage):
    _check(_lib.ceed_set_apply_variant(mesh.handle, op, prec, ne, stage))


def ceed_jacobi_diagonal(mesh: Mesh, op, qdata, prec, diag, flags=0, stream=None):
    _check(_lib.ceed_jacobi_diagonal(mesh.handle, op, _ptr(qdata), prec, _ptr(diag), flags, _stream(stream)))


def ceed_manufactured_rhs(mesh: Mesh, coeff_kind, b, flags=0, stream=None):
    _check(_lib.ceed_manufactured_rhs(mesh.handle, coeff_kind, _ptr(b), flags, _stream(stream)))


def _cg_opts(**kw):
    o = _CgOpts()
    for k, v in kw.items():
        if k == "qdata_lo":
            o.qdata_lo = _ptr(v)
        elif k == "pmg":
            o.pmg = v.handle if v is not None else None
        else:
            setattr(o, k, v)
    return o


def ceed_cg_workspace_bytes(mesh: Mesh, **opts) -> int:
    o = _cg_opts(**opts)
    return int(_lib.ceed_cg_workspace_bytes(mesh.handle, ctypes.byref(o)))


def ceed_cg_solve(mesh: Mesh, qdata, prec, b, x, work=None, stream=None, raise_on_error=True, **opts):
    """Returns (status, report dict).  opts are ceed_cg_opts fields (mode, tol, max_iter, ...)."""
    o = _cg_opts(**opts)
    nbytes = int(_lib.ceed_cg_workspace_bytes(mesh.handle, ctypes.byref(o)))
    if work is None:
        work = torch.empty(nbytes, dtype=torch.uint8, device=b.device)
    rep = _CgReport()
    st = _lib.ceed_cg_solve(mesh.handle, _ptr(qdata), prec, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(rep),
                            _ptr(work), work.numel() * work.element_size(), _stream(stream))
    report = dict(iterations=rep.iterations, outer_iterations=rep.outer_iterations,
                  rel_residual=rep.rel_residual, seconds=rep.seconds, fused=rep.fused)
    if raise_on_error and st not in (CEED_OK,):
        raise CeedError(st, _lib.ceed_last_error().decode())
    return st, report


class Batch:
    """Owns a ceed_batch_t and keeps its meshes and buffers alive."""

    def __init__(self, handle, keep):
        self.handle, self._keep = handle, keep

    def close(self):
        if self.handle:
            _lib.ceed_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_batch_create(meshes, qdata, prec, op, xs, ys, nrhs=1) -> Batch:
    n = len(meshes)
    arr = lambda items: (ctypes.c_void_p * n)(*items)
    h = ctypes.c_void_p()
    _check(_lib.ceed_batch_create(n, arr([m.handle for m in meshes]), arr([_ptr(q).value for q in qdata]), prec, op,
                                  arr([_ptr(x).value for x in xs]), arr([_ptr(y).value for y in ys]), nrhs,
                                  ctypes.byref(h)))
    return Batch(h, (list(meshes), list(qdata), list(xs), list(ys)))


def ceed_batch_apply(batch: Batch, stream=None):
    _check(_lib.ceed_batch_apply(batch.handle, _stream(stream)))


def ceed_batch_autotune(batch: Batch, stream=None) -> float:
    ms = ctypes.c_float()
    _check(_lib.ceed_batch_autotune(batch.handle, ctypes.byref(ms), _stream(stream)))
    return ms.value


def ceed_batch_info(batch: Batch):
    t, st, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint32()
    _check(_lib.ceed_batch_info(batch.handle, ctypes.byref(t), ctypes.byref(st), ctypes.byref(g)))
    return t.value, st.value, g.value


def ceed_batch_status(batch: Batch, stream=None):
    _check(_lib.ceed_batch_status(batch.handle, _stream(stream)))


def ceed_batch_destroy(batch: Batch):
    batch.close()


def ceed_mesh_status(mesh: Mesh, stream=None):
    _check(_lib.ceed_mesh_status(mesh.handle, _stream(stream)))


def ceed_set_wait_limits(copy_polls: int = -1, barrier_polls: int = -1):
    _check(_lib.ceed_set_wait_limits(copy_polls, barrier_polls))


def ceed_fma_throughput(kind: int, stream=None):
    """(TFLOP/s, FMAs per clock per SM, SM MHz) of kind 0 = FP64, 1 = FP32, 2 = FP32x2 FMA chains."""
    tf, per_clk, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.ceed_fma_throughput(kind, ctypes.byref(tf), ctypes.byref(per_clk), ctypes.byref(mhz), _stream(stream)))
    return tf.value, per_clk.value, mhz.value


class Pmg:
    """Owns a ceed_pmg_t and keeps its level meshes and quadrature data alive."""

    def __init__(self, handle, keep):
        self.handle, self._keep = handle, keep

    def close(self):
        if self.handle:
            _lib.ceed_pmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_pmg_create(meshes, qdata64, qdata_lo=None, prec_lo=CEED_F32, smooth_degree=0, smooth_ratio=0.0,
                    eig_iters=0, coarse_tol=0.0, coarse_max_iter=0, smoother=0, smoother_coeff=CEED_COEFF_SINE,
                    stream=None) -> Pmg:
    """smoother 0: Chebyshev-Jacobi; 1: Chebyshev on the overlapping Schwarz smoother."""
    n = len(meshes)
    arr = lambda items: (ctypes.c_void_p * n)(*items)
    lo = arr([_ptr(q).value if q is not None else None for q in qdata_lo]) if qdata_lo is not None else None
    o = _PmgOpts(smooth_degree, smooth_ratio, eig_iters, coarse_tol, coarse_max_iter, prec_lo, smoother,
                 smoother_coeff)
    h = ctypes.c_void_p()
    _check(_lib.ceed_pmg_create(n, arr([m.handle for m in meshes]), arr([_ptr(q).value for q in qdata64]), lo,
                                ctypes.byref(o), ctypes.byref(h), _stream(stream)))
    return Pmg(h, (list(meshes), list(qdata64), qdata_lo))


def ceed_pmg_vcycle(pmg: Pmg, r, z, stream=None):
    _check(_lib.ceed_pmg_vcycle(pmg.handle, _ptr(r), _ptr(z), _stream(stream)))


def ceed_pmg_prolong(pmg: Pmg, level, uc, uf, stream=None):
    _check(_lib.ceed_pmg_prolong(pmg.handle, level, _ptr(uc), _ptr(uf), _stream(stream)))


def ceed_pmg_restrict(pmg: Pmg, level, rf, rc, stream=None):
    _check(_lib.ceed_pmg_restrict(pmg.handle, level, _ptr(rf), _ptr(rc), _stream(stream)))


def ceed_pmg_info(pmg: Pmg, level) -> float:
    lam = ctypes.c_double()
    _check(_lib.ceed_pmg_info(pmg.handle, level, ctypes.byref(lam)))
    return lam.value


def ceed_pmg_destroy(pmg: Pmg):
    pmg.close()


def ceed_build_geometry(mesh: Mesh, geo, stream=None):
    _check(_lib.ceed_build_geometry(mesh.handle, _ptr(geo), _stream(stream)))


def ceed_apply_diffusion_k(mesh: Mesh, k, geo, x, y, flags=0, stream=None):
    _check(_lib.ceed_apply_diffusion_k(mesh.handle, _ptr(k), _ptr(geo), _ptr(x), _ptr(y), flags, _stream(stream)))


def ceed_apply_diffusion_adjoint(mesh: Mesh, k, geo, x, r, dLdx, dLdk, flags=0, stream=None):
    _check(_lib.ceed_apply_diffusion_adjoint(mesh.handle, _ptr(k), _ptr(geo), _ptr(x), _ptr(r), _ptr(dLdx),
                                             _ptr(dLdk), flags, _stream(stream)))


def ceed_simplex_sizes(p: int, q: int):
    """(P, Q) of the degree-p tetrahedron with q conical-rule points per direction."""
    P, Q = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ceed_simplex_sizes(p, q, ctypes.byref(P), ctypes.byref(Q)))
    return P.value, Q.value


def ceed_simplex_basis(p: int, q: int):
    """Host tables of the degree-p tetrahedron: interp [Q, P], grad [3, Q, P], qweight [Q], qref [Q, 3]."""
    import numpy as np
    P, Q = ceed_simplex_sizes(p, q)
    interp, grad = np.empty((Q, P)), np.empty((3, Q, P))
    qw, qref = np.empty(Q), np.empty((Q, 3))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_lib.ceed_simplex_basis(p, q, ptr(interp), ptr(grad), ptr(qw), ptr(qref)))
    return interp, grad, qw, qref


def ceed_hp_prolongation(nx: int, ny: int, nz: int, orders):
    """The conforming prolongation of an hp lattice, built on the host: (n_true, row_ptr, col, val, dirichlet)."""
    import numpy as np
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(-1))
    if o.size != nx * ny * nz:
        raise ValueError("one order per element")
    nt, nr, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    optr = o.ctypes.data_as(ctypes.c_void_p)
    _check(_lib.ceed_hp_prolongation(nx, ny, nz, optr, ctypes.byref(nt), ctypes.byref(nr), ctypes.byref(nnz),
                                     None, None, None, None))
    rp, col = np.empty(nr.value + 1, dtype=np.int64), np.empty(nnz.value, dtype=np.int64)
    val, d = np.empty(nnz.value), np.empty(nt.value, dtype=np.uint8)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_lib.ceed_hp_prolongation(nx, ny, nz, optr, ctypes.byref(nt), ctypes.byref(nr), ctypes.byref(nnz),
                                     ptr(rp), ptr(col), ptr(val), ptr(d)))
    return nt.value, rp, col, val, d


def ceed_schwarz_fdm_1d(p: int):
    """The Schwarz smoother's 1D fast-diagonalization basis in FP64: (S [P, P], lambda [P])."""
    import numpy as np
    S, lam = np.empty((p + 1, p + 1)), np.empty(p + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_lib.ceed_schwarz_fdm_1d(p, S.ctypes.data_as(dp), lam.ctypes.data_as(dp)))
    return S, lam


class NonTensor:
    """Owns a ceed_nt_t (non-tensor element operator); released on close() or garbage collection."""

    def __init__(self, handle, n_elem, n_ldof, P, Q):
        self.handle, self.n_elem, self.n_ldof, self.P, self.Q = handle, n_elem, n_ldof, P, Q

    def close(self):
        if self.handle:
            _lib.ceed_nt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_nt_setup(n_elem, n_ldof, interp, grad, qweight, qref, elem_dofs, vertices, dirichlet=None,
                  stream=None) -> NonTensor:
    """interp/grad/qweight/qref: host numpy float64 arrays; elem_dofs/vertices/dirichlet: CUDA tensors."""
    import numpy as np
    assert elem_dofs.dtype == torch.int32 and vertices.dtype == torch.float64
    assert dirichlet is None or dirichlet.dtype == torch.uint8
    interp, grad, qweight, qref = (np.ascontiguousarray(a, dtype=np.float64) for a in (interp, grad, qweight, qref))
    Q, P = interp.shape
    assert grad.shape == (3, Q, P) and qweight.shape == (Q,) and qref.shape == (Q, 3)
    hp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    d = _NtDesc(n_elem, n_ldof, P, Q, hp(interp), hp(grad), hp(qweight), hp(qref), _ptr(elem_dofs), _ptr(vertices),
                _ptr(dirichlet))
    h = ctypes.c_void_p()
    _check(_lib.ceed_nt_setup(ctypes.byref(d), ctypes.byref(h), _stream(stream)))
    return NonTensor(h, n_elem, n_ldof, P, Q)


def ceed_nt_destroy(nt: NonTensor):
    nt.close()


def ceed_nt_qdata_bytes(nt: NonTensor, op: int, prec: int) -> int:
    return int(_lib.ceed_nt_qdata_bytes(nt.handle, op, prec))


def alloc_nt_qdata(nt: NonTensor, op: int, prec: int, device=None) -> torch.Tensor:
    return torch.empty(ceed_nt_qdata_bytes(nt, op, prec), dtype=torch.uint8, device=device or "cuda")


def ceed_nt_build_qdata(nt: NonTensor, op, coeff_kind, coeff, prec, qdata, stream=None):
    if coeff_kind == CEED_COEFF_CONST:
        cval = (ctypes.c_double * 1)(float(coeff))
        cptr = ctypes.cast(cval, ctypes.c_void_p)
    else:
        cptr = _ptr(coeff) if coeff is not None else None
    _check(_lib.ceed_nt_build_qdata(nt.handle, op, coeff_kind, cptr, prec, _ptr(qdata), _stream(stream)))


def ceed_nt_apply(nt: NonTensor, op, qdata, prec, x, y, flags=0, stream=None):
    _check(_lib.ceed_nt_apply(nt.handle, op, _ptr(qdata), prec, _ptr(x), _ptr(y), flags, _stream(stream)))


def ceed_nt_set_algorithm(nt: NonTensor, op, prec, algo, eta=0, gemm_mode=0):
    _check(_lib.ceed_nt_set_algorithm(nt.handle, op, prec, algo, eta, gemm_mode))


def ceed_nt_get_algorithm(nt: NonTensor, op, prec):
    """(algo, eta, gemm_mode, ms) in use for (op, prec)."""
    a, e, g, ms = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_float()
    _check(_lib.ceed_nt_get_algorithm(nt.handle, op, prec, ctypes.byref(a), ctypes.byref(e), ctypes.byref(g),
                                      ctypes.byref(ms)))
    return a.value, e.value, g.value, ms.value


def ceed_nt_autotune(nt: NonTensor, op, qdata, prec, x, y, include_tf32=False, stream=None):
    _check(_lib.ceed_nt_autotune(nt.handle, op, _ptr(qdata), prec, _ptr(x), _ptr(y), int(include_tf32),
                                 _stream(stream)))
    return ceed_nt_get_algorithm(nt, op, prec)


def ceed_nt_status(nt: NonTensor, stream=None):
    _check(_lib.ceed_nt_status(nt.handle, _stream(stream)))


class Schwarz:
    """Owns a ceed_schwarz_t and keeps its mesh alive."""

    def __init__(self, handle, mesh):
        self.handle, self._mesh = handle, mesh

    def close(self):
        if self.handle:
            _lib.ceed_schwarz_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_schwarz_create(mesh: Mesh, coeff_kind=CEED_COEFF_SINE, coeff=None, stream=None) -> Schwarz:
    cptr = None
    if coeff_kind == CEED_COEFF_CONST:
        cval = (ctypes.c_double * 1)(float(coeff))
        cptr = ctypes.cast(cval, ctypes.c_void_p)
    h = ctypes.c_void_p()
    _check(_lib.ceed_schwarz_create(mesh.handle, coeff_kind, cptr, ctypes.byref(h), _stream(stream)))
    return Schwarz(h, mesh)


def ceed_schwarz_apply(sw: Schwarz, r, z, flags=0, stream=None):
    _check(_lib.ceed_schwarz_apply(sw.handle, _ptr(r), _ptr(z), flags, _stream(stream)))


def ceed_schwarz_destroy(sw: Schwarz):
    sw.close()


class Hp:
    """Owns a ceed_hp_t (conforming variable-order space and operator)."""

    def __init__(self, handle):
        self.handle = handle
        nt, nr, ng = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.ceed_hp_info(handle, ctypes.byref(nt), ctypes.byref(nr), ctypes.byref(ng)))
        self.n_true, self.n_rows, self.n_groups = nt.value, nr.value, ng.value

    def close(self):
        if self.handle:
            _lib.ceed_hp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ceed_hp_setup(nx, ny, nz, orders, vertices, q_rule=CEED_QRULE_GLL, dirichlet=True, stream=None) -> Hp:
    """orders: host int array [nx ny nz]; vertices: CUDA float64 tensor [E, 8, 3]."""
    import numpy as np
    o = np.ascontiguousarray(orders, dtype=np.int32)
    assert o.size == nx * ny * nz and vertices.dtype == torch.float64
    d = _HpDesc(nx, ny, nz, o.ctypes.data_as(ctypes.c_void_p), _ptr(vertices), q_rule, int(bool(dirichlet)))
    h = ctypes.c_void_p()
    _check(_lib.ceed_hp_setup(ctypes.byref(d), ctypes.byref(h), _stream(stream)))
    return Hp(h)


def ceed_hp_destroy(hp: Hp):
    hp.close()


def ceed_hp_info(hp: Hp):
    return hp.n_true, hp.n_rows, hp.n_groups


def ceed_hp_build_qdata(hp: Hp, op, coeff_kind, coeff=None, prec=CEED_F64, stream=None):
    if coeff_kind == CEED_COEFF_CONST:
        cval = (ctypes.c_double * 1)(float(coeff))
        cptr = ctypes.cast(cval, ctypes.c_void_p)
    else:
        cptr = None
    _check(_lib.ceed_hp_build_qdata(hp.handle, op, coeff_kind, cptr, prec, _stream(stream)))


def ceed_hp_prolong(hp: Hp, x, u_elem, stream=None):
    _check(_lib.ceed_hp_prolong(hp.handle, _ptr(x), _ptr(u_elem), _stream(stream)))


def ceed_hp_apply(hp: Hp, op, prec, x, y, flags=0, stream=None):
    _check(_lib.ceed_hp_apply(hp.handle, op, prec, _ptr(x), _ptr(y), flags, _stream(stream)))


def ceed_dot_workspace_bytes(n: int) -> int:
    return int(_lib.ceed_dot_workspace_bytes(n))


def ceed_dot(x, y, out, work, stream=None):
    _check(_lib.ceed_dot(_ptr(x), _ptr(y), x.numel(), _ptr(out), _ptr(work), _stream(stream)))


def ceed_dot_noalloc_max_n() -> int:
    return int(_lib.ceed_dot_noalloc_max_n())


def ceed_dot_noalloc(x, y, out, stream=None):
    """Dot product with no device allocation and no workspace (static scratch inside the library).

    For callers that cannot allocate device memory themselves; see include/ceed_gb300.h for the
    size limit (n <= ceed_dot_noalloc_max_n()) and the rule that calls must not overlap on the GPU.
    """
    _check(_lib.ceed_dot_noalloc(_ptr(x), _ptr(y), x.numel(), _ptr(out), _stream(stream)))


def ceed_last_error() -> str:
    return _lib.ceed_last_error().decode()


class DiffusionK(torch.autograd.Function):
    """y = A(k) x with a per-point coefficient k [E, Q^3]; backward runs the fused adjoint kernel.

    grad_x = A(k) grad_y (A is symmetric), grad_k[e, q] = (grad_xi g)_q^T Ghat_q (grad_xi x)_q with
    g = grad_y.  geo: stored geometry (ceed_build_geometry) or None to recompute it from the vertices.
    df: both passes in the FP64-accurate double-float arithmetic (stored geometry only).
    """

    @staticmethod
    def forward(ctx, x, k, mesh, geo, df=False):
        y = torch.empty_like(x)
        ctx.flags = CEED_APPLY_F64_DF if df else 0
        ceed_apply_diffusion_k(mesh, k, geo, x, y, flags=ctx.flags)
        ctx.save_for_backward(x, k)
        ctx.mesh, ctx.geo = mesh, geo
        return y

    @staticmethod
    def backward(ctx, gy):
        x, k = ctx.saved_tensors
        gy = gy.contiguous()
        gx = torch.empty_like(x)
        gk = torch.empty_like(k)
        ceed_apply_diffusion_adjoint(ctx.mesh, k, ctx.geo, x, gy, gx, gk, flags=ctx.flags)
        return gx, gk, None, None, None


def diffusion_k(x, k, mesh, geo=None, df=False):
    return DiffusionK.apply(x, k, mesh, geo, df)

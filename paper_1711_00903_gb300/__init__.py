"""GB300-native element-local tensor-product operators BP1.0, BP3.5 and
BP3.0 of high-order hexahedral spectral elements (Swirydowicz, Chalmers,
Karakus & Warburton, arXiv:1711.00903, Section 4).

This package is a thin ctypes binding over the C ABI in include/fem.h
(libfem.so, hand-written CUDA for sm_103a).  The functions keep the C
names; they only check and marshal arguments (device tensors, sizes, the
current torch stream).  Every step of the computation runs in the
library's kernels: there is no CPU path, and a call on tensors that are
not CUDA float64 tensors raises.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import _build

__all__ = [
    "FemError", "lib", "Basis", "fem_version", "fem_basis_setup", "fem_basis_free",
    "fem_basis_tables", "fem_basis_host_tables", "fem_mesh_geofacs", "fem_bp1_apply",
    "fem_bp35_apply", "fem_bp30_apply", "FEM_GEO_BP1", "FEM_GEO_BP35", "FEM_GEO_BP30",
    "geo_shape", "fem_mesh_geofacs_set", "fem_wait_timeouts", "fem_wait_selftest", "fem_layout_check", "fem_bp30_apply_layout", "fem_fma_probe",
    "FEM_LAYOUT_LINES", "FEM_LAYOUT_POINTS", "FEM_LAYOUT_WARP", "FEM_LAYOUT_STREAM", "fem_bp30_apply_f32_layout", "fem_bp35_apply_layout", "FEM_BATCH_POINTS30",
    "FEM_BATCH_POINTS35", "fem_bp35_apply_f32", "fem_bp30_apply_f32", "fem_bp30_apply_tc", "fem_bp35_apply_tc", "FEM_PREC_F16TC", "fem_stream_sum", "fem_bp35_jacobi", "fem_bp30_jacobi", "fem_dot", "fem_dot_scratch_size", "Pcg",
    "fem_bp35_apply_ex", "fem_bp30_apply_ex", "fem_bp1_bp30_apply", "FEM_PREC_F64", "FEM_PREC_F32", "FEM_PREC_F16G",
    "fem_pcg_create", "fem_pcg_solve", "fem_pcg_destroy", "FEM_ETIMEDOUT", "FEM_ECANCELED", "FEM_FAULT_WAIT_TIMEOUT", "FEM_EBREAKDOWN", "FEM_PCG_FP64", "FEM_PCG_MIXED", "FEM_PCG_MIXED16", "FEM_PCG_MIXED_TC", "fem_bp35_apply_f16g", "fem_bp30_apply_f16g",
    "Batch", "fem_batch_create", "FEM_OP_BP35", "FEM_OP_BP30", "Server",
    "FEM_REQ_QUEUED", "FEM_REQ_RUNNING", "FEM_REQ_DONE", "FEM_REQ_FAILED", "FEM_SERVE_FIFO", "FEM_SERVE_SHORTEST",
]

FEM_OK, FEM_EINVAL, FEM_ECUDA, FEM_ENOMEM, FEM_ENODEV = 0, -1, -2, -3, -4
FEM_EBREAKDOWN, FEM_ENOCONV, FEM_ETOOBIG, FEM_ETIMEDOUT, FEM_ECANCELED = -5, -6, -7, -8, -9
FEM_FAULT_WAIT_TIMEOUT = 1
FEM_PCG_FP64, FEM_PCG_MIXED, FEM_PCG_MIXED16, FEM_PCG_MIXED_TC = 0, 1, 2, 3
FEM_GEO_BP1, FEM_GEO_BP35, FEM_GEO_BP30 = 1, 2, 3
FEM_OP_BP35, FEM_OP_BP30 = 2, 3
FEM_LAYOUT_LINES, FEM_LAYOUT_POINTS, FEM_LAYOUT_WARP, FEM_LAYOUT_STREAM = 0, 1, 2, 3
FEM_BATCH_POINTS30, FEM_BATCH_POINTS35 = 1, 2
FEM_PREC_F64, FEM_PREC_F32, FEM_PREC_F16G, FEM_PREC_F16TC = 0, 1, 2, 3
FEM_REQ_QUEUED, FEM_REQ_RUNNING, FEM_REQ_DONE, FEM_REQ_FAILED = 0, 1, 2, 3
FEM_SERVE_FIFO, FEM_SERVE_SHORTEST = 0, 1
MAX_N = 15

_lock = threading.Lock()
_lib = None


class PcgOpts(C.Structure):
    """fem_pcg_opts (include/fem.h)."""
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int), ("check_every", C.c_int)]


class PcgInfo(C.Structure):
    """fem_pcg_info (include/fem.h)."""
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("relres", C.c_double)]


class BatchItem(C.Structure):
    """fem_batch_item (include/fem.h)."""
    _fields_ = [("op", C.c_int), ("basis", C.c_void_p), ("E", C.c_int64), ("geo", C.c_void_p),
                ("lam", C.c_double), ("q", C.c_void_p), ("out", C.c_void_p)]


class BatchConfig(C.Structure):
    """fem_batch_config (include/fem.h)."""
    _fields_ = [("threads", C.c_int), ("group", C.c_int), ("order", C.c_int), ("layout", C.c_int),
                ("ms", C.c_float)]


class ServeOpts(C.Structure):
    """fem_serve_opts (include/fem.h)."""
    _fields_ = [("hbm_budget", C.c_int64), ("max_active", C.c_int), ("check_every", C.c_int),
                ("policy", C.c_int), ("max_wait_s", C.c_double)]


class ServeRequest(C.Structure):
    """fem_serve_request (include/fem.h)."""
    _fields_ = [("op", C.c_int), ("N", C.c_int), ("E", C.c_int64), ("verts", C.c_void_p),
                ("rhs", C.c_void_p), ("x", C.c_void_p), ("lam", C.c_double), ("mode", C.c_int),
                ("tol", C.c_double)]


class ServeResult(C.Structure):
    """fem_serve_result (include/fem.h)."""
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("iters", C.c_int), ("outer", C.c_int),
                ("relres", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("bytes", C.c_int64)]


class FemError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {lib().fem_strerror(code).decode()}"
        if code in (FEM_ECUDA, FEM_ENODEV):
            msg += f" ({lib().fem_last_cuda_error().decode()})"
        super().__init__(msg)


def lib():
    """The loaded libfem.so (built in-tree with nvcc on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            i32, i64, dbl, vp, dp = C.c_int, C.c_int64, C.c_double, C.c_void_p, C.c_void_p
            L.fem_version.restype = i32
            L.fem_strerror.argtypes = [i32]
            L.fem_strerror.restype = C.c_char_p
            L.fem_last_cuda_error.restype = C.c_char_p
            L.fem_basis_setup.argtypes = [i32, C.POINTER(vp)]
            L.fem_basis_free.argtypes = [vp]
            L.fem_basis_free.restype = None
            L.fem_basis_degree.argtypes = [vp]
            L.fem_basis_tables.argtypes = [vp] + [dp] * 7
            L.fem_basis_host_tables.argtypes = [i32] + [dp] * 7
            L.fem_mesh_geofacs.argtypes = [vp, i32, i64, dp, dp, dp, vp]
            L.fem_bp1_apply.argtypes = [vp, i64, dp, dp, dp, vp]
            L.fem_bp35_apply.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp30_apply.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp35_apply_f32.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp30_apply_f32.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp30_apply_tc.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp35_apply_tc.argtypes = [vp, i64, dp, dbl, dp, dp, vp]
            L.fem_bp30_apply_f32_layout.argtypes = [vp, i64, dp, dbl, dp, dp, i32, vp]
            L.fem_bp35_apply_layout.argtypes = [vp, i64, dp, dbl, dp, dp, i32, vp]
            L.fem_stream_sum.argtypes = [i32, i64, dp, dp, i32, vp]
            L.fem_mesh_geofacs_set.argtypes = [vp, i64, dp, dp, dp, dp, vp]
            L.fem_wait_timeouts.argtypes = [C.POINTER(C.c_ulonglong), i32]
            L.fem_fma_probe_threads.restype = i64
            L.fem_wait_selftest.argtypes = [C.POINTER(C.c_ulonglong)]
            L.fem_layout_check.argtypes = [C.POINTER(C.c_int64)]
            L.fem_fma_probe.argtypes = [i64, dp, vp]
            L.fem_bp30_apply_layout.argtypes = [vp, i64, dp, dbl, dp, dp, i32, vp]
            L.fem_bp35_apply_f16g.argtypes = [vp, i64, dp, dp, dbl, dp, dp, vp]
            L.fem_bp30_apply_f16g.argtypes = [vp, i64, dp, dp, dbl, dp, dp, vp]
            L.fem_bp35_apply_ex.argtypes = [vp, i64, i32, dp, dp, dbl, dp, dp, vp]
            L.fem_bp1_bp30_apply.argtypes = [vp, i64, dp, dbl, dp, dp, dp, vp]
            L.fem_bp30_apply_ex.argtypes = [vp, i64, i32, dp, dp, dbl, dp, dp, vp]
            L.fem_bp35_jacobi.argtypes = [vp, i64, dp, dbl, dp, vp]
            L.fem_dot_scratch_size.restype = i64
            L.fem_dot.argtypes = [i64, dp, dp, dp, dp, vp]
            L.fem_pcg_create.argtypes = [vp, i32, i64, dp, dbl, i32, C.POINTER(vp)]
            L.fem_bp30_jacobi.argtypes = [vp, i64, dp, dbl, dp, vp]
            L.fem_bp30_jacobi.restype = i32
            L.fem_pcg_solve.argtypes = [vp, dp, dp, C.POINTER(PcgOpts), C.POINTER(PcgInfo), vp]
            L.fem_dot_noalloc_max_n.restype = i64
            L.fem_dot_noalloc.argtypes = [i64, dp, dp, dp, vp]
            L.fem_dot_noalloc.restype = i32
            L.fem_batch_create.argtypes = [C.POINTER(BatchItem), i32, C.POINTER(vp)]
            L.fem_batch_apply.argtypes = [vp, vp]
            L.fem_batch_tune.argtypes = [vp, vp, i32, C.POINTER(BatchConfig), i32, C.POINTER(i32)]
            L.fem_batch_get_config.argtypes = [vp, C.POINTER(BatchConfig)]
            L.fem_batch_set_config.argtypes = [vp, C.POINTER(BatchConfig)]
            L.fem_batch_graph_launch.argtypes = [vp, vp]
            L.fem_batch_destroy.argtypes = [vp]
            L.fem_batch_destroy.restype = None
            for f in ("fem_batch_create", "fem_batch_apply", "fem_batch_tune", "fem_batch_get_config",
                      "fem_batch_set_config", "fem_batch_graph_launch"):
                getattr(L, f).restype = i32
            L.fem_serve_create.argtypes = [C.POINTER(ServeOpts), C.POINTER(vp)]
            L.fem_serve_submit.argtypes = [vp, C.POINTER(ServeRequest), C.POINTER(i64)]
            L.fem_serve_progress.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
            L.fem_serve_poll.argtypes = [vp, i64, C.POINTER(ServeResult)]
            L.fem_serve_wait.argtypes = [vp, i64, dbl, C.POINTER(ServeResult)]
            L.fem_serve_wait.restype = i32
            L.fem_serve_cancel.argtypes = [vp, i64]
            L.fem_serve_cancel.restype = i32
            L.fem_serve_clock.argtypes = [vp]
            L.fem_serve_clock.restype = dbl
            L.fem_serve_in_use.argtypes = [vp]
            L.fem_serve_in_use.restype = i64
            L.fem_serve_destroy.argtypes = [vp]
            L.fem_serve_destroy.restype = None
            for f in ("fem_serve_create", "fem_serve_submit", "fem_serve_progress", "fem_serve_poll"):
                getattr(L, f).restype = i32
            L.fem_pcg_destroy.argtypes = [vp]
            L.fem_pcg_inject_fault.argtypes = [vp, i32]
            L.fem_pcg_inject_fault.restype = i32
            L.fem_pcg_destroy.restype = None
            for f in ("fem_basis_setup", "fem_basis_tables", "fem_basis_host_tables",
                      "fem_mesh_geofacs", "fem_bp1_apply", "fem_bp35_apply", "fem_bp30_apply",
                      "fem_basis_degree", "fem_mesh_geofacs_set", "fem_wait_timeouts", "fem_bp30_apply_layout", "fem_fma_probe",
                      "fem_bp35_apply_f16g", "fem_bp30_apply_f16g", "fem_bp35_apply_ex", "fem_bp30_apply_ex",
                      "fem_bp1_bp30_apply",
                      "fem_bp35_apply_f32", "fem_bp30_apply_f32", "fem_bp30_apply_tc", "fem_bp35_apply_tc", "fem_bp30_apply_f32_layout", "fem_bp35_apply_layout", "fem_stream_sum", "fem_bp35_jacobi", "fem_bp30_jacobi", "fem_dot",
                      "fem_pcg_create", "fem_pcg_solve"):
                getattr(L, f).restype = i32
            _lib = L
    return _lib


def _check(code: int, what: str):
    if code != FEM_OK:
        raise FemError(code, what)


def fem_version() -> int:
    return lib().fem_version()


class Basis:
    """Owning wrapper of a fem_basis handle of degree N."""

    def __init__(self, handle: int, N: int):
        self.handle = C.c_void_p(handle)
        self.N, self.n, self.m = N, N + 1, N + 2

    def free(self):
        if self.handle and self.handle.value:
            lib().fem_basis_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fem_basis_setup(N: int) -> Basis:
    """Degree-N basis on the current device (Section 4 tables; FP64)."""
    h = C.c_void_p()
    _check(lib().fem_basis_setup(int(N), C.byref(h)), f"fem_basis_setup(N={N})")
    return Basis(h.value, int(N))


def fem_basis_free(b: Basis):
    b.free()


def _tables(fn, *args, N):
    import numpy as np
    n, m = N + 1, N + 2
    out = {"r": np.zeros(n), "w": np.zeros(n), "rt": np.zeros(m), "wt": np.zeros(m),
           "I": np.zeros((m, n)), "D": np.zeros((n, n)), "Dt": np.zeros((m, m))}
    ptrs = [out[k].ctypes.data for k in ("r", "w", "rt", "wt", "I", "D", "Dt")]
    _check(fn(*args, *ptrs), "basis tables")
    return out


def fem_basis_tables(b: Basis) -> dict:
    """Host copies of r, w, rt, wt, I, D, Dt of a handle."""
    return _tables(lib().fem_basis_tables, b.handle, N=b.N)


def fem_basis_host_tables(N: int) -> dict:
    """The same tables computed on the host without a GPU."""
    if not 1 <= N <= MAX_N:
        raise ValueError("N must be in 1..15")
    return _tables(lib().fem_basis_host_tables, int(N), N=N)


def geo_shape(b: Basis, kind: int, E: int):
    if kind == FEM_GEO_BP1:
        return (E, b.m ** 3)
    if kind == FEM_GEO_BP35:
        return (E, 7, b.n ** 3)
    if kind == FEM_GEO_BP30:
        return (E, 7, b.m ** 3)
    raise ValueError("bad geometric-factor kind")


def _dev(t, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} entries, expected {numel}")
    return t.data_ptr()


def _stream(stream, device):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def fem_mesh_geofacs(b: Basis, kind: int, verts, geo=None, detJ_min=None, stream=None):
    """Geometric factors from element vertices (E, 8, 3) on the device.
    Returns geo (allocated when not given)."""
    import torch
    E = verts.shape[0] if verts.dim() else 0
    _dev(verts, "verts", E * 24)
    if geo is None:
        geo = torch.empty(geo_shape(b, kind, E), dtype=torch.float64, device=verts.device)
    shp = geo_shape(b, kind, E)
    _dev(geo, "geo", int(torch.Size(shp).numel()))
    dmin = _dev(detJ_min, "detJ_min", E) if detJ_min is not None else None
    _check(lib().fem_mesh_geofacs(b.handle, int(kind), E, verts.data_ptr(), geo.data_ptr(), dmin,
                                  _stream(stream, verts.device)), "fem_mesh_geofacs")
    return geo


def fem_mesh_geofacs_set(b: Basis, verts, wJ=None, G35=None, G30=None, stream=None):
    """The factors of the three operators of one mesh in one call (any
    subset; wJ and the BP3.0 factors share one kernel).  Outputs passed as
    None are not computed.  Returns (wJ, G35, G30)."""
    E = verts.shape[0] if verts.dim() else 0
    _dev(verts, "verts", E * 24)
    ptrs = []
    for t, kind, name in ((wJ, FEM_GEO_BP1, "wJ"), (G35, FEM_GEO_BP35, "G35"), (G30, FEM_GEO_BP30, "G30")):
        if t is None:
            ptrs.append(None)
        else:
            import torch
            _dev(t, name, int(torch.Size(geo_shape(b, kind, E)).numel()))
            ptrs.append(t.data_ptr())
    _check(lib().fem_mesh_geofacs_set(b.handle, E, verts.data_ptr(), *ptrs, _stream(stream, verts.device)),
           "fem_mesh_geofacs_set")
    return wJ, G35, G30


def _apply_out(q, out, b):
    import torch
    E = q.shape[0]
    _dev(q, "q", E * b.n ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev(out, "out", E * b.n ** 3)
    return E, out


def fem_bp1_apply(b: Basis, wJ, q, out=None, stream=None):
    """BP1.0 mass matvec Mq = I^T J I q (Algorithm 3)."""
    E, out = _apply_out(q, out, b)
    _dev(wJ, "wJ", E * b.m ** 3)
    _check(lib().fem_bp1_apply(b.handle, E, wJ.data_ptr(), q.data_ptr(), out.data_ptr(),
                               _stream(stream, q.device)), "fem_bp1_apply")
    return out


def fem_bp35_apply(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.5 matvec D^T G D q + lambda J q at the GLL nodes (Algorithm 4)."""
    E, out = _apply_out(q, out, b)
    _dev(G, "G", E * 7 * b.n ** 3)
    _check(lib().fem_bp35_apply(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                _stream(stream, q.device)), "fem_bp35_apply")
    return out


def fem_bp30_apply(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.0 matvec I^T (Dt^T G Dt + lambda J) I q (Algorithm 5)."""
    E, out = _apply_out(q, out, b)
    _dev(G, "G", E * 7 * b.m ** 3)
    _check(lib().fem_bp30_apply(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                _stream(stream, q.device)), "fem_bp30_apply")
    return out


def _dev32(t, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} entries, expected {numel}")
    return t.data_ptr()


def _apply_f16g(name, b: Basis, G16, ginv, lam, q, out, stream, gpts):
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    if not isinstance(G16, torch.Tensor) or not G16.is_cuda or G16.dtype != torch.float16 or \
            not G16.is_contiguous() or G16.numel() != E * 7 * gpts:
        raise TypeError("G16 must be a contiguous float16 CUDA tensor of E*7*points values")
    if not isinstance(ginv, torch.Tensor) or not ginv.is_cuda or ginv.dtype != torch.float64 or ginv.numel() != 1:
        raise TypeError("ginv must be a one-element float64 CUDA tensor")
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(getattr(lib(), name)(b.handle, E, G16.data_ptr(), ginv.data_ptr(), float(lam), q.data_ptr(),
                                out.data_ptr(), _stream(stream, q.device)), name)
    return out


def fem_bp35_apply_f16g(b: Basis, G16, ginv, lam: float, q, out=None, stream=None):
    """BP3.5 matvec with binary16 factors (float16 tensor) and FP32 data;
    the output is multiplied by ginv (one-element float64 device tensor)."""
    return _apply_f16g("fem_bp35_apply_f16g", b, G16, ginv, lam, q, out, stream, b.n ** 3)


def fem_bp30_apply_f16g(b: Basis, G16, ginv, lam: float, q, out=None, stream=None):
    """BP3.0 matvec with binary16 factors and FP32 data (see fem_bp35_apply_f16g)."""
    return _apply_f16g("fem_bp30_apply_f16g", b, G16, ginv, lam, q, out, stream, b.m ** 3)


def _apply_ex(name, b: Basis, prec, G, lam, q, ginv, out, stream, gpts):
    import torch
    if prec not in (FEM_PREC_F64, FEM_PREC_F32, FEM_PREC_F16G, FEM_PREC_F16TC):
        raise ValueError(f"unknown precision {prec}")
    E = q.shape[0]
    vec = _dev if prec == FEM_PREC_F64 else _dev32
    vec(q, "q", E * b.n ** 3)
    gptr = None
    if prec == FEM_PREC_F16G:
        if not isinstance(G, torch.Tensor) or not G.is_cuda or G.dtype != torch.float16 or \
                not G.is_contiguous() or G.numel() != E * 7 * gpts:
            raise TypeError("G must be a contiguous float16 CUDA tensor of E*7*points values")
        if not isinstance(ginv, torch.Tensor) or not ginv.is_cuda or ginv.dtype != torch.float64 or \
                ginv.numel() != 1:
            raise TypeError("ginv must be a one-element float64 CUDA tensor")
        gptr = ginv.data_ptr()
    else:
        vec(G, "G", E * 7 * gpts)
    if out is None:
        out = torch.empty_like(q)
    vec(out, "out", E * b.n ** 3)
    _check(getattr(lib(), name)(b.handle, E, int(prec), G.data_ptr(), gptr, float(lam), q.data_ptr(),
                                out.data_ptr(), _stream(stream, q.device)), name)
    return out


def fem_bp35_apply_ex(b: Basis, prec: int, G, lam: float, q, ginv=None, out=None, stream=None):
    """BP3.5 matvec with the precision chosen at run time: FEM_PREC_F64
    (float64 G, q), FEM_PREC_F32 (float32 G, q) or FEM_PREC_F16G (float16 G
    scaled by a power of two undone by ginv, float32 q)."""
    return _apply_ex("fem_bp35_apply_ex", b, prec, G, lam, q, ginv, out, stream, b.n ** 3)


def fem_bp30_apply_ex(b: Basis, prec: int, G, lam: float, q, ginv=None, out=None, stream=None):
    """BP3.0 matvec with the precision chosen at run time (see fem_bp35_apply_ex)."""
    return _apply_ex("fem_bp30_apply_ex", b, prec, G, lam, q, ginv, out, stream, b.m ** 3)


def fem_bp1_bp30_apply(b: Basis, G, lam: float, q, out_m=None, out_a=None, stream=None):
    """BP1.0 and BP3.0 of one field in one pass: returns (Mq, Aq), with
    BP1.0's wJ the seventh plane of the BP3.0 factors G."""
    E, out_a = _apply_out(q, out_a, b)
    _, out_m = _apply_out(q, out_m, b)
    _dev(G, "G", E * 7 * b.m ** 3)
    _check(lib().fem_bp1_bp30_apply(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out_m.data_ptr(),
                                    out_a.data_ptr(), _stream(stream, q.device)), "fem_bp1_bp30_apply")
    return out_m, out_a


def fem_bp30_apply_layout(b: Basis, G, lam: float, q, layout: int, out=None, stream=None):
    """BP3.0 matvec with a chosen thread layout (FEM_LAYOUT_LINES or
    FEM_LAYOUT_POINTS)."""
    E, out = _apply_out(q, out, b)
    _dev(G, "G", E * 7 * b.m ** 3)
    _check(lib().fem_bp30_apply_layout(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                       int(layout), _stream(stream, q.device)), "fem_bp30_apply_layout")
    return out


def fem_bp35_apply_layout(b: Basis, G, lam: float, q, layout: int, out=None, stream=None):
    """BP3.5 matvec with a chosen thread layout (FEM_LAYOUT_LINES or
    FEM_LAYOUT_POINTS: one thread per GLL node, Algorithm 7)."""
    E, out = _apply_out(q, out, b)
    _dev(G, "G", E * 7 * b.n ** 3)
    _check(lib().fem_bp35_apply_layout(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                       int(layout), _stream(stream, q.device)), "fem_bp35_apply_layout")
    return out


def fem_bp35_apply_f32(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.5 matvec in FP32 (FP32 factors and field)."""
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    _dev32(G, "G", E * 7 * b.n ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(lib().fem_bp35_apply_f32(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                    _stream(stream, q.device)), "fem_bp35_apply_f32")
    return out


def fem_wait_selftest():
    """Runs a kernel whose bounded wait cannot complete; returns (how many
    warps gave up, the call's status): (2, FEM_ETIMEDOUT) when the wait
    limit works and the kernel reported it through its status word."""
    c = C.c_ulonglong(0)
    code = lib().fem_wait_selftest(C.byref(c))
    if code not in (FEM_OK, FEM_ETIMEDOUT):
        _check(code, "fem_wait_selftest")
    return int(c.value), code


def fem_layout_check() -> int:
    """Host-side check of the kernels' shared-memory element boxes; returns
    the number of violations (0 when every layout holds)."""
    v = C.c_int64(-1)
    _check(lib().fem_layout_check(C.byref(v)), "fem_layout_check")
    return int(v.value)


def fem_fma_probe(iters: int, out=None, stream=None):
    """One launch of the FP64 issue-rate probe; returns (out, flops)."""
    import torch
    nt = int(lib().fem_fma_probe_threads())
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device="cuda")
    _dev(out, "out", nt)
    _check(lib().fem_fma_probe(int(iters), out.data_ptr(), _stream(stream, out.device)), "fem_fma_probe")
    return out, 2 * 8 * int(iters) * nt


def fem_wait_timeouts(reset: bool = False) -> int:
    """Bounded device-side waits that gave up (0 in normal operation)."""
    c = C.c_ulonglong(0)
    _check(lib().fem_wait_timeouts(C.byref(c), 1 if reset else 0), "fem_wait_timeouts")
    return int(c.value)


def fem_stream_sum(src, out=None, stream=None):
    """Roofline calibration stream: out = src.sum(0) over the planes of a
    (planes, n) float64 or float32 CUDA tensor, in plane order."""
    import torch
    if not isinstance(src, torch.Tensor) or not src.is_cuda or src.dim() != 2 or not src.is_contiguous() \
            or src.dtype not in (torch.float64, torch.float32):
        raise TypeError("src must be a contiguous 2-D float64/float32 CUDA tensor")
    planes, n = src.shape
    if out is None:
        out = torch.empty(n, dtype=src.dtype, device=src.device)
    if not out.is_cuda or out.dtype != src.dtype or out.numel() != n or not out.is_contiguous():
        raise TypeError("out must be a contiguous CUDA tensor of n values of src's dtype")
    _check(lib().fem_stream_sum(int(planes), int(n), src.data_ptr(), out.data_ptr(), src.element_size(),
                                _stream(stream, src.device)), "fem_stream_sum")
    return out


def fem_bp30_apply_f32(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.0 matvec in FP32 (FP32 factors and field)."""
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    _dev32(G, "G", E * 7 * b.m ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(lib().fem_bp30_apply_f32(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                    _stream(stream, q.device)), "fem_bp30_apply_f32")
    return out


def fem_bp30_apply_f32_layout(b: Basis, G, lam: float, q, layout: int, out=None, stream=None):
    """FP32 BP3.0 matvec by a chosen kernel (FEM_LAYOUT_LINES: the block
    kernel; FEM_LAYOUT_WARP: one warp per element)."""
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    _dev32(G, "G", E * 7 * b.m ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(lib().fem_bp30_apply_f32_layout(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                           int(layout), _stream(stream, q.device)), "fem_bp30_apply_f32_layout")
    return out


def fem_bp35_apply_tc(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.5 matvec with the derivative contractions on the tensor cores
    (FP32 factors and field, split f16 operands, FP32 accumulation)."""
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    _dev32(G, "G", E * 7 * b.n ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(lib().fem_bp35_apply_tc(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                   _stream(stream, q.device)), "fem_bp35_apply_tc")
    return out


def fem_bp30_apply_tc(b: Basis, G, lam: float, q, out=None, stream=None):
    """BP3.0 matvec with the contractions on the tensor cores (FP32 factors
    and field, split f16 operands, FP32 accumulation)."""
    import torch
    E = q.shape[0]
    _dev32(q, "q", E * b.n ** 3)
    _dev32(G, "G", E * 7 * b.m ** 3)
    if out is None:
        out = torch.empty_like(q)
    _dev32(out, "out", E * b.n ** 3)
    _check(lib().fem_bp30_apply_tc(b.handle, E, G.data_ptr(), float(lam), q.data_ptr(), out.data_ptr(),
                                   _stream(stream, q.device)), "fem_bp30_apply_tc")
    return out


def fem_bp30_jacobi(b: Basis, G, lam: float, out=None, stream=None):
    """Inverse diagonal of the BP3.0 operator (Jacobi preconditioner)."""
    import torch
    E = G.shape[0]
    _dev(G, "G", E * 7 * b.m ** 3)
    if out is None:
        out = torch.empty((E, b.n ** 3), dtype=torch.float64, device=G.device)
    _dev(out, "dinv", E * b.n ** 3)
    _check(lib().fem_bp30_jacobi(b.handle, E, G.data_ptr(), float(lam), out.data_ptr(),
                                 _stream(stream, G.device)), "fem_bp30_jacobi")
    return out


def fem_bp35_jacobi(b: Basis, G, lam: float, out=None, stream=None):
    """Inverse diagonal of the BP3.5 operator (Jacobi preconditioner)."""
    import torch
    E = G.shape[0]
    _dev(G, "G", E * 7 * b.n ** 3)
    if out is None:
        out = torch.empty((E, b.n ** 3), dtype=torch.float64, device=G.device)
    _dev(out, "dinv", E * b.n ** 3)
    _check(lib().fem_bp35_jacobi(b.handle, E, G.data_ptr(), float(lam), out.data_ptr(),
                                 _stream(stream, G.device)), "fem_bp35_jacobi")
    return out


def fem_dot_scratch_size() -> int:
    return int(lib().fem_dot_scratch_size())


def fem_dot(x, y, result=None, scratch=None, stream=None):
    """Deterministic FP64 dot product of two device vectors; returns the
    one-element device tensor holding it."""
    import torch
    n = x.numel()
    _dev(x, "x")
    _dev(y, "y", n)
    if result is None:
        result = torch.empty(1, dtype=torch.float64, device=x.device)
    if scratch is None:
        scratch = torch.empty(fem_dot_scratch_size(), dtype=torch.float64, device=x.device)
    _dev(result, "result")
    _dev(scratch, "scratch")
    if scratch.numel() < fem_dot_scratch_size():
        raise ValueError("scratch too small")
    _check(lib().fem_dot(n, x.data_ptr(), y.data_ptr(), result.data_ptr(), scratch.data_ptr(),
                         _stream(stream, x.device)), "fem_dot")
    return result


class Pcg:
    """Owning wrapper of a fem_pcg solver context."""

    def __init__(self, handle: int, basis: Basis, E: int, G):
        self.handle = C.c_void_p(handle)
        self.basis, self.E, self.G = basis, E, G  # keep G alive with the context

    def solve(self, rhs, x=None, tol=1e-10, maxit=0, inner_tol=0.0, inner_maxit=0, check_every=0,
              stream=None, raise_on_error=True):
        return fem_pcg_solve(self, rhs, x, tol, maxit, inner_tol, inner_maxit, check_every, stream,
                             raise_on_error)

    def inject_fault(self, fault=FEM_FAULT_WAIT_TIMEOUT):
        """Arms the host-side fault injection of the next solve
        (fem_pcg_inject_fault)."""
        _check(lib().fem_pcg_inject_fault(self.handle, int(fault)), "fem_pcg_inject_fault")

    def free(self):
        if self.handle and self.handle.value:
            lib().fem_pcg_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fem_pcg_create(b: Basis, G, lam: float, mode: int = FEM_PCG_FP64, op: int = FEM_OP_BP35) -> Pcg:
    """Jacobi-PCG solver context for the BP3.5 (op FEM_OP_BP35) or BP3.0
    (FEM_OP_BP30) system with factors G."""
    E = G.shape[0]
    _dev(G, "G", E * 7 * (b.n ** 3 if op == FEM_OP_BP35 else b.m ** 3))
    h = C.c_void_p()
    _check(lib().fem_pcg_create(b.handle, int(op), E, G.data_ptr(), float(lam), int(mode), C.byref(h)),
           "fem_pcg_create")
    return Pcg(h.value, b, E, G)


def fem_pcg_solve(s: Pcg, rhs, x=None, tol=1e-10, maxit=0, inner_tol=0.0, inner_maxit=0,
                  check_every=0, stream=None, raise_on_error=True):
    """Solves A x = rhs from the x passed in (zeros when None).  Returns
    (x, info dict, status code)."""
    import torch
    n = s.E * s.basis.n ** 3
    _dev(rhs, "rhs", n)
    if x is None:
        x = torch.zeros_like(rhs)
    _dev(x, "x", n)
    opts = PcgOpts(float(tol), int(maxit), float(inner_tol), int(inner_maxit), int(check_every))
    info = PcgInfo()
    code = lib().fem_pcg_solve(s.handle, rhs.data_ptr(), x.data_ptr(), C.byref(opts), C.byref(info),
                               _stream(stream, rhs.device))
    if raise_on_error and code not in (FEM_OK,):
        raise FemError(code, "fem_pcg_solve")
    return x, {"iters": info.iters, "outer": info.outer, "relres": info.relres}, code


def fem_pcg_destroy(s: Pcg):
    s.free()


class Batch:
    """Owning wrapper of a fem_batch: many meshes of mixed degree applied in
    one persistent launch.  items: list of (op, basis, geo, lam, q, out)."""

    def __init__(self, items):
        self.items = list(items)  # keeps every tensor and basis alive
        arr = (BatchItem * max(1, len(self.items)))()
        for k, (op, basis, geo, lam, q, out) in enumerate(self.items):
            E = q.shape[0]
            n, m = basis.n, basis.m
            _dev(q, "q", E * n ** 3)
            _dev(out, "out", E * n ** 3)
            _dev(geo, "geo", E * 7 * (n ** 3 if op == FEM_OP_BP35 else m ** 3))
            arr[k] = BatchItem(int(op), basis.handle.value, E, geo.data_ptr(), float(lam), q.data_ptr(),
                               out.data_ptr())
        h = C.c_void_p()
        _check(lib().fem_batch_create(arr, len(self.items), C.byref(h)), "fem_batch_create")
        self.handle = h

    def apply(self, stream=None):
        dev = self.items[0][4].device if self.items else None
        _check(lib().fem_batch_apply(self.handle, _stream(stream, dev)), "fem_batch_apply")

    def graph_launch(self, stream=None):
        dev = self.items[0][4].device if self.items else None
        _check(lib().fem_batch_graph_launch(self.handle, _stream(stream, dev)), "fem_batch_graph_launch")

    def tune(self, reps=5, stream=None):
        """Times every launch configuration; keeps the fastest.  Returns the
        list of (threads, group, order, layout, ms)."""
        dev = self.items[0][4].device if self.items else None
        res = (BatchConfig * 64)()
        cnt = C.c_int(0)
        _check(lib().fem_batch_tune(self.handle, _stream(stream, dev), int(reps), res, 64, C.byref(cnt)),
               "fem_batch_tune")
        return [(r.threads, r.group, r.order, r.layout, r.ms) for r in res[:cnt.value]]

    @property
    def config(self):
        c = BatchConfig()
        _check(lib().fem_batch_get_config(self.handle, C.byref(c)), "fem_batch_get_config")
        return {"threads": c.threads, "group": c.group, "order": c.order, "layout": c.layout, "ms": c.ms}

    @config.setter
    def config(self, cfg):
        c = BatchConfig(int(cfg["threads"]), int(cfg["group"]), int(cfg["order"]), int(cfg.get("layout", 0)), 0.0)
        _check(lib().fem_batch_set_config(self.handle, C.byref(c)), "fem_batch_set_config")

    def free(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().fem_batch_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fem_batch_create(items) -> Batch:
    return Batch(items)


class Server:
    """Owning wrapper of a fem_server (continuous batching of Helmholtz
    solves).  Host arrays of a request are kept referenced here until the
    request has finished."""

    def __init__(self, hbm_budget=120 << 30, max_active=8, check_every=8, policy=0, max_wait_s=0.0):
        """policy: FEM_SERVE_FIFO (0) or FEM_SERVE_SHORTEST (1); max_wait_s:
        the aging bound of FEM_SERVE_SHORTEST (0: the library's default)."""
        o = ServeOpts(int(hbm_budget), int(max_active), int(check_every), int(policy), float(max_wait_s))
        h = C.c_void_p()
        _check(lib().fem_serve_create(C.byref(o), C.byref(h)), "fem_serve_create")
        self.handle = h
        self._keep = {}

    def submit(self, op, N, verts, rhs, lam=1.0, mode=FEM_PCG_FP64, tol=1e-8):
        """Queues a solve; verts (E, 8, 3) and rhs (E, (N+1)^3) float64 host
        arrays.  Returns (id, x) with x the host array the solution lands in."""
        import numpy as np
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        E = verts.shape[0]
        if rhs.size != E * (N + 1) ** 3:
            raise ValueError("rhs size does not match E and N")
        x = np.zeros_like(rhs)
        r = ServeRequest(int(op), int(N), E, verts.ctypes.data, rhs.ctypes.data, x.ctypes.data, float(lam),
                         int(mode), float(tol))
        rid = C.c_int64()
        _check(lib().fem_serve_submit(self.handle, C.byref(r), C.byref(rid)), "fem_serve_submit")
        self._keep[rid.value] = (verts, rhs, x)
        return rid.value, x

    def progress(self):
        a, q = C.c_int(), C.c_int()
        _check(lib().fem_serve_progress(self.handle, C.byref(a), C.byref(q)), "fem_serve_progress")
        return a.value, q.value

    def poll(self, rid):
        r = ServeResult()
        _check(lib().fem_serve_poll(self.handle, int(rid), C.byref(r)), "fem_serve_poll")
        return {k: getattr(r, k) for k, _ in ServeResult._fields_}

    def wait(self, rid, timeout_s):
        """Progresses until request rid finishes or timeout_s passes; returns
        (result dict, status): FEM_OK, or FEM_ETIMEDOUT at the deadline."""
        r = ServeResult()
        code = lib().fem_serve_wait(self.handle, int(rid), float(timeout_s), C.byref(r))
        if code not in (FEM_OK, FEM_ETIMEDOUT):
            _check(code, "fem_serve_wait")
        return {k: getattr(r, k) for k, _ in ServeResult._fields_}, code

    def cancel(self, rid):
        _check(lib().fem_serve_cancel(self.handle, int(rid)), "fem_serve_cancel")

    def forget(self, rid):
        """Drops this wrapper's references to a finished request's host
        arrays (the caller keeps its own x if it needs it)."""
        self._keep.pop(int(rid), None)

    def clock(self) -> float:
        return lib().fem_serve_clock(self.handle)

    def in_use(self) -> int:
        return lib().fem_serve_in_use(self.handle)

    def drain(self, poll_sleep=0.0):
        """Progresses until nothing is queued or in flight."""
        import time
        while True:
            a, q = self.progress()
            if a == 0 and q == 0:
                return
            if poll_sleep:
                time.sleep(poll_sleep)

    def free(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().fem_serve_destroy(self.handle)
            self.handle = C.c_void_p(None)
        self._keep = {}

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

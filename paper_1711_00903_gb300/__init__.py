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
    "geo_shape",
]

FEM_OK, FEM_EINVAL, FEM_ECUDA, FEM_ENOMEM, FEM_ENODEV = 0, -1, -2, -3, -4
FEM_GEO_BP1, FEM_GEO_BP35, FEM_GEO_BP30 = 1, 2, 3
MAX_N = 15

_lock = threading.Lock()
_lib = None


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
            for f in ("fem_basis_setup", "fem_basis_tables", "fem_basis_host_tables",
                      "fem_mesh_geofacs", "fem_bp1_apply", "fem_bp35_apply", "fem_bp30_apply",
                      "fem_basis_degree"):
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

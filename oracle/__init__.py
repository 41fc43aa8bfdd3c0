"""Plain FP64 CPU oracle for BP1.0 / BP3.5 / BP3.0 (arXiv:1711.00903).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the bench's
CPU-baseline leg are the only callers.  The product path (the CUDA library
and its binding) never imports this package.

The arithmetic lives in ``fem_oracle.c`` (plain C, IEEE double, no
fast-math); this module compiles it with gcc on first use and wraps it with
ctypes.  Every function below names the passage of the paper it follows.
Parity status: every function here is pinned by the CPU tests
(tests/test_oracle_*.py) against closed forms, library routines, brute-force
element matrices and exact-integration invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfem_oracle.so")
_lock = threading.Lock()
_lib = None

MAXN = 15

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile fem_oracle.c into oracle/_build/libfem_oracle.so (gcc, -O2,
    OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
            "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            L.or_set_threads.argtypes = [i32]
            L.or_set_threads.restype = i32
            L.or_gauss.argtypes = [i32, _dp, _dp]
            L.or_gll.argtypes = [i32, _dp, _dp]
            L.or_basis.argtypes = [i32] + [_dp] * 7
            L.or_lagrange_row.argtypes = [i32, _dp, dbl, _dp]
            L.or_lagrange_d1_row.argtypes = [i32, _dp, dbl, _dp]
            L.or_map.argtypes = [_dp, dbl, dbl, dbl, _dp, _dp]
            L.or_map.restype = None
            L.or_geofacs_grid.argtypes = [i32, _dp, _dp, i32, i64, _dp, _dp]
            L.or_geofacs_grid.restype = dbl
            L.or_geofacs.argtypes = [i32, i32, i64, _dp, _dp]
            L.or_geofacs.restype = dbl
            L.or_bp1.argtypes = [i32, i64, _dp, _dp, _dp]
            L.or_bp35.argtypes = [i32, i64, _dp, dbl, _dp, _dp]
            L.or_bp30.argtypes = [i32, i64, _dp, dbl, _dp, _dp]
            L.or_dense_element.argtypes = [i32, i32, i32, dbl, _dp, _dp]
            L.or_bp35_diag.argtypes = [i32, i64, _dp, dbl, _dp]
            L.or_pcg_bp35.argtypes = [i32, i64, _dp, dbl, _dp, _dp, dbl, i32,
                                      C.POINTER(C.c_double)]
            L.or_bp30_diag.argtypes = [i32, i64, _dp, dbl, _dp]
            L.or_pcg_bp30.argtypes = [i32, i64, _dp, dbl, _dp, _dp, dbl, i32,
                                      C.POINTER(C.c_double)]
            _lib = L
    return _lib


def set_threads(t: int) -> int:
    """OpenMP threads for the element loops; returns the count in use."""
    return lib().or_set_threads(int(t))


def gauss(m: int):
    """m-point Gauss-Legendre nodes and weights (Section 4, GL rule)."""
    x, w = np.zeros(m), np.zeros(m)
    assert lib().or_gauss(m, x, w) == 0
    return x, w


def gll(N: int):
    """N+1 point Gauss-Lobatto-Legendre nodes and weights (Section 4)."""
    x, w = np.zeros(N + 1), np.zeros(N + 1)
    assert lib().or_gll(N, x, w) == 0
    return x, w


class Basis:
    """r, w (GLL), rt, wt (Gauss), I (m x n), D (n x n), Dt (m x m) of
    degree N (Table of notation; eq. interpolationOps, derivativeOps)."""

    def __init__(self, N: int):
        if not 1 <= N <= MAXN:
            raise ValueError("N must be in 1..15")
        n, m = N + 1, N + 2
        self.N, self.n, self.m = N, n, m
        self.r, self.w = np.zeros(n), np.zeros(n)
        self.rt, self.wt = np.zeros(m), np.zeros(m)
        self.I, self.D, self.Dt = np.zeros((m, n)), np.zeros((n, n)), np.zeros((m, m))
        assert lib().or_basis(N, self.r, self.w, self.rt, self.wt,
                              self.I, self.D, self.Dt) == 0


def lagrange_row(nodes, x):
    """l_i(x) for every Lagrange polynomial on `nodes` (product formula)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    out = np.zeros(len(nodes))
    lib().or_lagrange_row(len(nodes), nodes, float(x), out)
    return out


def lagrange_d1_row(nodes, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    out = np.zeros(len(nodes))
    lib().or_lagrange_d1_row(len(nodes), nodes, float(x), out)
    return out


def trilinear(verts8, r, s, t):
    """x(r,s,t) and X = dx/d(r,s,t) of one element's trilinear map."""
    v = np.ascontiguousarray(verts8, dtype=np.float64).reshape(24)
    x, X = np.zeros(3), np.zeros(9)
    lib().or_map(v, float(r), float(s), float(t), x, X)
    return x, X.reshape(3, 3)


KIND_BP1, KIND_BP35, KIND_BP30 = 1, 2, 3


def geo_points(N: int, kind: int) -> int:
    q = N + 1 if kind == KIND_BP35 else N + 2
    return q ** 3


def geofacs(N: int, kind: int, verts: np.ndarray):
    """Geometric factors (Section 4: G^e and J^e with quadrature weights).
    kind 1: (E, m^3) wJ at Gauss points; 2: (E, 7, n^3) at GLL nodes;
    3: (E, 7, m^3) at Gauss points.  Returns (geo, min detJ)."""
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    E = verts.shape[0]
    P = geo_points(N, kind)
    geo = np.zeros((E, P) if kind == KIND_BP1 else (E, 7, P))
    mindet = lib().or_geofacs(N, kind, E, verts.reshape(-1), geo.reshape(-1))
    return geo, mindet


def geofacs_grid(nodes, weights, kind: int, verts: np.ndarray):
    """Geometric factors on an arbitrary tensor grid (used by the tests)."""
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    q, E = len(nodes), verts.shape[0]
    geo = np.zeros((E, q ** 3) if kind == KIND_BP1 else (E, 7, q ** 3))
    mindet = lib().or_geofacs_grid(q, nodes, weights, kind, E, verts.reshape(-1),
                                   geo.reshape(-1))
    return geo, mindet


def _vec(a, E, P):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != E * P:
        raise ValueError("bad size")
    return a.reshape(-1)


def bp1(N: int, wJ: np.ndarray, q: np.ndarray) -> np.ndarray:
    """BP1.0 mass matvec Mq = I^T J I q per element (Algorithm 3)."""
    n, m = N + 1, N + 2
    E = q.shape[0]
    out = np.zeros((E, n ** 3))
    assert lib().or_bp1(N, E, _vec(wJ, E, m ** 3), _vec(q, E, n ** 3), out.reshape(-1)) == 0
    return out


def bp35(N: int, geo: np.ndarray, lam: float, q: np.ndarray) -> np.ndarray:
    """BP3.5 collocated screened Poisson D^T G D q + lambda J q (Algorithm 4)."""
    n = N + 1
    E = q.shape[0]
    out = np.zeros((E, n ** 3))
    assert lib().or_bp35(N, E, _vec(geo, E, 7 * n ** 3), float(lam),
                         _vec(q, E, n ** 3), out.reshape(-1)) == 0
    return out


def bp30(N: int, geo: np.ndarray, lam: float, q: np.ndarray) -> np.ndarray:
    """BP3.0 dealiased screened Poisson I^T (Dt^T G Dt + lambda J) I q
    (Algorithm 5)."""
    n, m = N + 1, N + 2
    E = q.shape[0]
    out = np.zeros((E, n ** 3))
    assert lib().or_bp30(N, E, _vec(geo, E, 7 * m ** 3), float(lam),
                         _vec(q, E, n ** 3), out.reshape(-1)) == 0
    return out


def dense_element(N: int, verts8: np.ndarray, rule: str, stiff: bool, lam: float = 0.0):
    """Brute-force element matrix from the quadrature sums of Section 4
    (eq. massQuad / stiffQuad / stiffQuad2), no sum factorisation.
    rule 'gauss' (N+2 points) or 'gll' (N+1 points)."""
    n = N + 1
    A = np.zeros((n ** 3, n ** 3))
    v = np.ascontiguousarray(verts8, dtype=np.float64).reshape(24)
    assert lib().or_dense_element(N, 1 if rule == "gll" else 0, int(stiff), float(lam), v,
                                  A.reshape(-1)) == 0
    return A


def bp35_diag(N: int, geo: np.ndarray, lam: float) -> np.ndarray:
    """Closed-form diagonal of the BP3.5 operator (Algorithm 4's D^T G D +
    lambda J), the Jacobi preconditioner."""
    n = N + 1
    E = geo.shape[0]
    out = np.zeros((E, n ** 3))
    assert lib().or_bp35_diag(N, E, _vec(geo, E, 7 * n ** 3), float(lam), out.reshape(-1)) == 0
    return out


def pcg_bp35(N: int, geo: np.ndarray, lam: float, b: np.ndarray, x0=None, tol=1e-10, maxit=10000):
    """Jacobi-PCG (Saad, Algorithm 9.1) on the unassembled BP3.5 system
    A x = b.  Returns (x, iterations, relative residual); raises on
    breakdown."""
    n = N + 1
    E = b.shape[0]
    x = np.zeros((E, n ** 3)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rel = C.c_double(0.0)
    it = lib().or_pcg_bp35(N, E, _vec(geo, E, 7 * n ** 3), float(lam), _vec(b, E, n ** 3),
                           x.reshape(-1), float(tol), int(maxit), C.byref(rel))
    if it < 0:
        raise RuntimeError(f"oracle PCG failed ({it})")
    return x, it, rel.value


def bp30_diag(N: int, geo: np.ndarray, lam: float) -> np.ndarray:
    """Diagonal of the BP3.0 operator (Algorithm 5's I^T (Dt^T G Dt +
    lambda J) I), entry by entry from the gradients of the basis functions
    at the Gauss points."""
    n, m = N + 1, N + 2
    E = geo.shape[0]
    out = np.zeros((E, n ** 3))
    assert lib().or_bp30_diag(N, E, _vec(geo, E, 7 * m ** 3), float(lam), out.reshape(-1)) == 0
    return out


def pcg_bp30(N: int, geo: np.ndarray, lam: float, b: np.ndarray, x0=None, tol=1e-10, maxit=10000):
    """Jacobi-PCG (Saad, Algorithm 9.1) on the unassembled BP3.0 system."""
    n, m = N + 1, N + 2
    E = b.shape[0]
    x = np.zeros((E, n ** 3)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rel = C.c_double(0.0)
    it = lib().or_pcg_bp30(N, E, _vec(geo, E, 7 * m ** 3), float(lam), _vec(b, E, n ** 3),
                           x.reshape(-1), float(tol), int(maxit), C.byref(rel))
    if it < 0:
        raise RuntimeError(f"oracle PCG failed ({it})")
    return x, it, rel.value


def gll_node_coordinates(N: int, verts: np.ndarray) -> np.ndarray:
    """Physical coordinates (E, n^3, 3) of every element's GLL nodes under
    its trilinear map (used to build manufactured right-hand sides)."""
    r, _ = gll(N)
    n = N + 1
    E = verts.shape[0]
    out = np.zeros((E, n ** 3, 3))
    for e in range(E):
        p = 0
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    out[e, p], _ = trilinear(verts[e], r[i], r[j], r[k])
                    p += 1
    return out

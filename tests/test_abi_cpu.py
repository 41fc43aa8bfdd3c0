"""CPU checks of the C ABI: the library builds and loads, exports every
function include/fem.h declares, its host-side basis agrees with the
oracle's, and argument errors are reported before any GPU work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_1711_00903_gb300 as fem

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fem.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fem_basis_setup", "fem_basis_free", "fem_mesh_geofacs", "fem_bp1_apply",
                 "fem_bp35_apply", "fem_bp30_apply"):
        assert must in names


@pytest.mark.parametrize("name", _declared())
def test_library_exports_symbol(name):
    assert hasattr(fem.lib(), name), name


def test_shared_memory_box_layouts_hold():
    """The element boxes the operator kernels lay out in shared memory
    (FP64 and the FP32 layouts chosen against bank conflicts, every degree)
    map each point to a distinct word inside its buffer, and the swizzled
    FP32 BP3.5 boxes (N = 7, 15) serve the lines of every direction, taken
    by the 32 lanes of a warp, without a bank conflict.  A host-side check
    in the library: no GPU."""
    assert fem.fem_layout_check() == 0
    with pytest.raises(TypeError):
        fem.fem_layout_check(1)


def test_version_and_strerror():
    L = fem.lib()
    assert fem.fem_version() >= 10000
    for code in (0, -1, -2, -3, -4):
        assert L.fem_strerror(code)
    assert b"unknown" in L.fem_strerror(-99)


@pytest.mark.parametrize("N", range(1, 16))
def test_host_basis_matches_oracle(N):
    """The library's basis (eigenvalue route, barycentric formulas) and the
    oracle's (Newton on Legendre, product formulas) are independent codes."""
    t = fem.fem_basis_host_tables(N)
    b = oracle.Basis(N)
    for k, ref in (("r", b.r), ("w", b.w), ("rt", b.rt), ("wt", b.wt)):
        np.testing.assert_allclose(t[k], ref, rtol=0, atol=2e-15)
    np.testing.assert_allclose(t["I"], b.I, rtol=0, atol=1e-14)
    scale = N * N
    np.testing.assert_allclose(t["D"], b.D, rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(t["Dt"], b.Dt, rtol=0, atol=1e-14 * scale)


def test_host_tables_reject_bad_degree():
    L = fem.lib()
    z = np.zeros(400)
    for N in (0, 16, -3):
        assert L.fem_basis_host_tables(N, *([z.ctypes.data] * 7)) == fem.FEM_EINVAL


def test_argument_errors_need_no_gpu():
    L = fem.lib()
    p = C.c_void_p(4096)  # never dereferenced: every call below fails its checks first
    assert L.fem_basis_setup(0, C.byref(C.c_void_p())) == fem.FEM_EINVAL
    assert L.fem_basis_setup(16, C.byref(C.c_void_p())) == fem.FEM_EINVAL
    assert L.fem_basis_setup(3, None) == fem.FEM_EINVAL
    assert L.fem_bp1_apply(None, 1, p, p, p, None) == fem.FEM_EINVAL
    assert L.fem_bp35_apply(None, 1, p, 1.0, p, p, None) == fem.FEM_EINVAL
    assert L.fem_bp30_apply(None, 1, p, 1.0, p, p, None) == fem.FEM_EINVAL
    assert L.fem_bp1_bp30_apply(None, 1, p, 1.0, p, p, p, None) == fem.FEM_EINVAL
    for prec in (fem.FEM_PREC_F64, fem.FEM_PREC_F32, fem.FEM_PREC_F16G, 3, -1):
        assert L.fem_bp35_apply_ex(None, 1, prec, p, p, 1.0, p, p, None) == fem.FEM_EINVAL
        assert L.fem_bp30_apply_ex(None, 1, prec, p, p, 1.0, p, p, None) == fem.FEM_EINVAL
    assert L.fem_mesh_geofacs(None, 1, 1, p, p, None, None) == fem.FEM_EINVAL
    assert L.fem_basis_degree(None) == fem.FEM_EINVAL
    assert L.fem_basis_tables(None, *([None] * 7)) == fem.FEM_EINVAL
    L.fem_basis_free(None)  # accepted
    bad = fem.ServeOpts(1 << 30, 4, 8, 7)  # unknown admission policy
    assert L.fem_serve_create(C.byref(bad), C.byref(C.c_void_p())) == fem.FEM_EINVAL
    assert L.fem_bp35_apply_f32(None, 1, p, 1.0, p, p, None) == fem.FEM_EINVAL
    assert L.fem_bp30_apply_f32(None, 1, p, 1.0, p, p, None) == fem.FEM_EINVAL
    # calibration stream: plane count, word size, vector alignment, overlap
    a, b = C.c_void_p(1 << 20), C.c_void_p(1 << 24)
    assert L.fem_stream_sum(0, 64, a, b, 8, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(33, 64, a, b, 8, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(2, 64, a, b, 2, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(2, 3, a, b, 8, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(2, 64, C.c_void_p((1 << 20) + 8), b, 8, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(2, 64, a, C.c_void_p((1 << 20) + 512), 8, None) == fem.FEM_EINVAL
    assert L.fem_stream_sum(2, 0, a, b, 8, None) == 0  # nothing to do
    assert L.fem_mesh_geofacs_set(None, 1, p, p, None, None, None) == fem.FEM_EINVAL
    assert L.fem_bp30_apply_layout(None, 1, p, 1.0, p, p, fem.FEM_LAYOUT_POINTS, None) == fem.FEM_EINVAL
    assert L.fem_bp30_apply_layout(None, 1, p, 1.0, p, p, 7, None) == fem.FEM_EINVAL


def test_binding_refuses_host_tensors():
    torch = pytest.importorskip("torch")
    fake = fem.Basis(0, 3)
    q = torch.zeros(2, 64, dtype=torch.float64)
    with pytest.raises(TypeError):
        fem.fem_bp35_apply(fake, torch.zeros(2, 7, 64, dtype=torch.float64), 1.0, q)
    with pytest.raises(TypeError):
        fem.fem_bp1_apply(fake, torch.zeros(2, 125, dtype=torch.float64), q)

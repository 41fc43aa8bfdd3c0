"""The allocation-free dot product (fem_dot_noalloc) through the C ABI.

It serves callers that cannot allocate device memory where they need a
reduction (a serving loop with a fixed memory budget, an application-owned
allocator): its partial sums live in a device array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes alone in a fresh process (the first call performs the one-time
device set-up)."""
import ctypes as C

import numpy as np
import pytest

import fem_synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _noalloc(L, x, y, out, stream=0):
    return L.fem_dot_noalloc(x.numel(), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                             C.c_void_p(out.data_ptr()), C.c_void_p(stream))


@pytest.mark.parametrize("n", [0, 1, 8191, 8193, 3_000_001])
def test_matches_allocating_entry_point_twice(n):
    import torch
    import paper_1711_00903_gb300 as fem
    L = fem.lib()
    x = _dev(fem_synth.field(31, 1, max(n, 1))[0][:n])
    y = _dev(fem_synth.field(32, 1, max(n, 1))[0][:n])
    ref = fem.fem_dot(x, y).item()
    scale = float((x * y).abs().sum().item()) if n else 1.0
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share and reuse the library's scratch
        out.fill_(float("nan"))
        assert _noalloc(L, x, y, out) == fem.FEM_OK
        torch.cuda.synchronize()
        got = out.item()
        assert abs(got - ref) <= 1e-12 * scale


def test_rejects_sizes_beyond_the_scratch_capacity():
    import torch
    import paper_1711_00903_gb300 as fem
    L = fem.lib()
    cap = L.fem_dot_noalloc_max_n()
    assert cap == 4096 * 8192
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # pointers are never dereferenced: the size check comes first
    assert L.fem_dot_noalloc(cap + 1, C.c_void_p(16), C.c_void_p(16), C.c_void_p(out.data_ptr()),
                             None) == fem.FEM_ETOOBIG
    assert L.fem_dot_noalloc(-1, None, None, C.c_void_p(out.data_ptr()), None) == fem.FEM_EINVAL
    assert b"capacity" in L.fem_strerror(fem.FEM_ETOOBIG)

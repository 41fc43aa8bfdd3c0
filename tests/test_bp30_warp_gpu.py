"""GPU parity of the FP32 BP3.0 kernels selectable through
fem_bp30_apply_f32_layout (FEM_LAYOUT_LINES: the block kernel;
FEM_LAYOUT_STREAM: the TMA stream kernel with one factor stage;
FEM_LAYOUT_WARP: one warp per element) through the C ABI, against the FP64
oracle applied to the same FP32-rounded factors and field, and against each
other.  Bar: the FP32 operators' 2e-6 (N + 2) in the relative max norm."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref)
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.fixture(scope="module")
def bases():
    import paper_1711_00903_gb300 as fem
    return {N: fem.fem_basis_setup(N) for N in range(1, 16)}


@pytest.mark.parametrize("N", range(1, 16))
@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_bp30_warp_parity(bases, N, lam):
    import torch
    import paper_1711_00903_gb300 as fem
    b, E = bases[N], 37
    v = fem_synth.box_mesh(4, 4, 4, jitter=0.1)[:E].copy()
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP30, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    got = fem.fem_bp30_apply_f32_layout(b, g32, lam, q32, fem.FEM_LAYOUT_WARP).cpu().numpy()
    ref = oracle.bp30(N, g32.cpu().numpy().astype(np.float64), lam, q32.cpu().numpy().astype(np.float64))
    assert _rel(got, ref) <= 2e-6 * (N + 2)
    blk = fem.fem_bp30_apply_f32_layout(b, g32, lam, q32, fem.FEM_LAYOUT_LINES).cpu().numpy()
    assert _rel(got, blk) <= 4e-6 * (N + 2)


def test_bp30_warp_layout_argument(bases):
    import torch
    import paper_1711_00903_gb300 as fem
    b = bases[3]
    g = torch.zeros((2, 7 * 125), dtype=torch.float32, device="cuda")
    q = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        fem.fem_bp30_apply_f32_layout(b, g, 1.0, q, 7)


@pytest.mark.parametrize("N", range(1, 16))
def test_bp30_stream_parity(bases, N):
    """The stream kernel on a ragged mesh whose elements outnumber the
    persistent grid several times over (every block walks several elements,
    stages reused), against the oracle and the block kernel; at a degree
    where an element does not fit in shared memory the layout is refused."""
    import torch
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    E = 2000 if N <= 7 else 400
    v = fem_synth.box_mesh(13, 13, 12, jitter=0.1)[:E].copy()
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP30, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    try:
        got = fem.fem_bp30_apply_f32_layout(b, g32, 1.0, q32, fem.FEM_LAYOUT_STREAM)
    except fem.FemError:
        assert N >= 14  # 7 m^3 factors, the field stages and three boxes exceed 227 KB
        return
    pick = np.unique(np.concatenate([np.arange(0, E, max(1, E // 40)), [E - 1]]))
    tp = torch.from_numpy(pick).cuda()
    ref = oracle.bp30(N, g32[tp].cpu().numpy().astype(np.float64), 1.0, q32[tp].cpu().numpy().astype(np.float64))
    assert _rel(got[tp].cpu().numpy(), ref) <= 2e-6 * (N + 2)
    blk = fem.fem_bp30_apply_f32_layout(b, g32, 1.0, q32, fem.FEM_LAYOUT_LINES)
    assert ((got - blk).abs().max() / blk.abs().max()).item() <= 4e-6 * (N + 2)
    assert fem.fem_wait_timeouts() == 0

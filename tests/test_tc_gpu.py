"""GPU parity of the tensor-core BP3.0 and BP3.5 operators
(fem_bp30_apply_tc, fem_bp35_apply_tc: split f16 mma.sync contractions with
FP32 accumulation, FP32 factors and field) through the C ABI, against the
FP64 oracle applied to the same FP32-rounded factors and field.

Tolerance.  Each contraction carries x_hi Op_hi + x_lo Op_hi + x_hi Op_lo,
which leaves about 3 * 2^-22 of the line's largest term per contraction,
and each of the nine stored stages rounds to FP32; the bound used here is
the FP32 CUDA-core operator's, 2e-6 (N + 2) in the relative max norm (the
line sums grow with the contraction length)."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref)
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    return np.abs(got - ref).max() / np.abs(ref).max()


def _tol(N):
    return 2e-6 * (N + 2)


@pytest.fixture(scope="module")
def bases():
    import paper_1711_00903_gb300 as fem
    return {N: fem.fem_basis_setup(N) for N in range(1, 16)}


def _case(fem, b, N, E, seed=fem_synth.SEED_MESH):
    import torch
    v = fem_synth.box_mesh(4, 4, 4, jitter=0.1, seed=seed)[:E].copy()
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP30, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    return g32, q32


@pytest.mark.parametrize("N", range(1, 16))
@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_bp30_tc_parity(bases, N, lam):
    """N = 1..15 on a ragged 37-element jittered mesh, lambda 0 and 1."""
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    g32, q32 = _case(fem, b, N, 37)
    got = fem.fem_bp30_apply_tc(b, g32, lam, q32).cpu().numpy()
    ref = oracle.bp30(N, g32.cpu().numpy().astype(np.float64), lam, q32.cpu().numpy().astype(np.float64))
    assert _rel(got, ref) <= _tol(N)


@pytest.mark.parametrize("N", [1, 2, 5, 7, 8, 9, 10, 13, 15])
def test_bp30_tc_matches_fp32_operator(bases, N):
    """Same inputs through the FP32 CUDA-core operator: both within the bar
    of the oracle, so within twice the bar of each other."""
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    g32, q32 = _case(fem, b, N, 64)
    tc = fem.fem_bp30_apply_tc(b, g32, 1.0, q32).cpu().numpy()
    f32 = fem.fem_bp30_apply_f32(b, g32, 1.0, q32).cpu().numpy()
    assert _rel(tc, f32) <= 2 * _tol(N)


@pytest.mark.parametrize("N", [3, 7, 12])
def test_bp30_tc_power_of_two_scaling_is_exact(bases, N):
    """Every line is scaled by a power of two before the f16 split and
    unscaled after: the operator of 2^k q is 2^k times the operator of q bit
    for bit, from 2^-100 to 2^100 (far outside the f16 range)."""
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    g32, q32 = _case(fem, b, N, 20)
    base = fem.fem_bp30_apply_tc(b, g32, 1.0, q32)
    for k in (-100, -30, -7, 9, 40, 100):
        got = fem.fem_bp30_apply_tc(b, g32, 1.0, q32 * 2.0 ** k)
        assert bool((got == base * 2.0 ** k).all()), k


@pytest.mark.parametrize("N", [2, 7, 11])
def test_bp30_tc_mixed_magnitudes(bases, N):
    """A field whose elements span 2^-60 .. 2^60 in magnitude (each element
    scaled by its own power of two): every element keeps the accuracy of
    the bar relative to its own size."""
    import torch
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    E = 25
    g32, q32 = _case(fem, b, N, E)
    sc = torch.tensor([2.0 ** (5 * (e % 25) - 60) for e in range(E)], device="cuda", dtype=torch.float32)
    qs = q32 * sc[:, None]
    got = fem.fem_bp30_apply_tc(b, g32, 1.0, qs).cpu().numpy()
    ref = oracle.bp30(N, g32.cpu().numpy().astype(np.float64), 1.0, qs.cpu().numpy().astype(np.float64))
    for e in range(E):
        assert _rel(got[e], ref[e]) <= _tol(N), e


def test_bp30_tc_empty_single_and_arguments(bases):
    import torch
    import paper_1711_00903_gb300 as fem
    b = bases[4]
    g32, q32 = _case(fem, b, 4, 1)
    got = fem.fem_bp30_apply_tc(b, g32, 1.0, q32).cpu().numpy()
    ref = oracle.bp30(4, g32.cpu().numpy().astype(np.float64), 1.0, q32.cpu().numpy().astype(np.float64))
    assert _rel(got, ref) <= _tol(4)
    e0 = torch.empty((0, 125), dtype=torch.float32, device="cuda")
    assert fem.fem_bp30_apply_tc(b, torch.empty((0, 7 * 216), dtype=torch.float32, device="cuda"), 1.0,
                                 e0).shape == (0, 125)
    with pytest.raises(Exception):  # output aliasing the input
        fem.fem_bp30_apply_tc(b, g32, 1.0, q32, out=q32)


def test_bp30_tc_full_size_sampled(bases):
    """N = 7 on the 32^3 benchmark mesh (E = 32768), 48 sampled elements
    against the oracle, and every element against the FP32 operator."""
    import torch
    import paper_1711_00903_gb300 as fem
    N, b = 7, bases[7]
    v = fem_synth.box_mesh(32)
    E = v.shape[0]
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP30, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    out = fem.fem_bp30_apply_tc(b, g32, 1.0, q32)
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([rng.choice(E, 46, replace=False), [0, E - 1]]))
    tp = torch.from_numpy(pick).cuda()
    ref = oracle.bp30(N, g32[tp].cpu().numpy().astype(np.float64), 1.0, q32[tp].cpu().numpy().astype(np.float64))
    assert _rel(out[tp].cpu().numpy(), ref) <= _tol(N)
    f32 = fem.fem_bp30_apply_f32(b, g32, 1.0, q32)
    assert ((out - f32).abs().max() / f32.abs().max()).item() <= 2 * _tol(N)


def _case35(fem, b, N, E, seed=fem_synth.SEED_MESH):
    import torch
    v = fem_synth.box_mesh(4, 4, 4, jitter=0.1, seed=seed)[:E].copy()
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP35, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    return g32, q32


@pytest.mark.parametrize("N", range(1, 16))
@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_bp35_tc_parity(bases, N, lam):
    """BP3.5 on the tensor cores, N = 1..15 on a ragged 37-element mesh,
    against the oracle and the FP32 CUDA-core operator."""
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    g32, q32 = _case35(fem, b, N, 37)
    got = fem.fem_bp35_apply_tc(b, g32, lam, q32).cpu().numpy()
    ref = oracle.bp35(N, g32.cpu().numpy().astype(np.float64), lam, q32.cpu().numpy().astype(np.float64))
    assert _rel(got, ref) <= _tol(N)
    f32 = fem.fem_bp35_apply_f32(b, g32, lam, q32).cpu().numpy()
    assert _rel(got, f32) <= 2 * _tol(N)


@pytest.mark.parametrize("N", [2, 7, 13])
def test_bp35_tc_power_of_two_scaling_is_exact(bases, N):
    import paper_1711_00903_gb300 as fem
    b = bases[N]
    g32, q32 = _case35(fem, b, N, 20)
    base = fem.fem_bp35_apply_tc(b, g32, 1.0, q32)
    for k in (-100, -9, 30, 100):
        assert bool((fem.fem_bp35_apply_tc(b, g32, 1.0, q32 * 2.0 ** k) == base * 2.0 ** k).all()), k


def test_bp35_tc_full_size_sampled(bases):
    """N = 7 on the 32^3 benchmark mesh, 48 sampled elements against the
    oracle and every element against the FP32 operator."""
    import torch
    import paper_1711_00903_gb300 as fem
    N, b = 7, bases[7]
    v = fem_synth.box_mesh(32)
    E = v.shape[0]
    g32 = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP35, torch.from_numpy(v).cuda()).float()
    q32 = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).cuda().float()
    out = fem.fem_bp35_apply_tc(b, g32, 1.0, q32)
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([rng.choice(E, 46, replace=False), [0, E - 1]]))
    tp = torch.from_numpy(pick).cuda()
    ref = oracle.bp35(N, g32[tp].cpu().numpy().astype(np.float64), 1.0, q32[tp].cpu().numpy().astype(np.float64))
    assert _rel(out[tp].cpu().numpy(), ref) <= _tol(N)
    f32 = fem.fem_bp35_apply_f32(b, g32, 1.0, q32)
    assert ((out - f32).abs().max() / f32.abs().max()).item() <= 2 * _tol(N)

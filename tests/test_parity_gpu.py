"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle:
geometric factors and the BP1.0 / BP3.5 / BP3.0 operators for every degree
N = 1..15, ragged element counts, both lambda branches, empty and single
element inputs, and the full-size 32^3 mesh on sampled elements.

Bar: ||y_gpu - y_oracle||_inf / ||y_oracle||_inf <= 1e-12 (FP64)."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _torch():
    import torch
    return torch


def _fem():
    import paper_1711_00903_gb300 as fem
    return fem


def _rel(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    return np.abs(got - ref).max() / np.abs(ref).max()


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _mesh(E, jitter=0.1, nx=4, ny=4, nz=4, seed=fem_synth.SEED_MESH):
    v = fem_synth.box_mesh(nx, ny, nz, jitter=jitter, seed=seed)
    assert E <= v.shape[0]
    return v[:E].copy()


E_RAGGED = 37  # not a multiple of any elements-per-block choice


@pytest.fixture(scope="module")
def bases():
    fem = _fem()
    return {N: fem.fem_basis_setup(N) for N in range(1, 16)}


@pytest.mark.parametrize("N", range(1, 16))
def test_basis_tables_device_handle(bases, N):
    fem = _fem()
    t = fem.fem_basis_tables(bases[N])
    b = oracle.Basis(N)
    np.testing.assert_allclose(t["I"], b.I, rtol=0, atol=1e-14)
    np.testing.assert_allclose(t["D"], b.D, rtol=0, atol=1e-14 * N * N)


@pytest.mark.parametrize("kind", [1, 2, 3], ids=["bp1", "bp35", "bp30"])
@pytest.mark.parametrize("N", range(1, 16))
def test_geofacs_parity(bases, N, kind):
    fem, torch = _fem(), _torch()
    v = _mesh(E_RAGGED)
    ref, mindet = oracle.geofacs(N, kind, v)
    dmin = torch.full((E_RAGGED,), float("nan"), dtype=torch.float64, device="cuda")
    geo = fem.fem_mesh_geofacs(bases[N], kind, _dev(v), detJ_min=dmin)
    torch.cuda.synchronize()
    got = geo.cpu().numpy()
    if kind == 1:
        assert _rel(got, ref) < TOL
    else:
        for g in range(7):
            assert _rel(got[:, g], ref[:, g]) < TOL, f"plane {g}"
    assert abs(dmin.min().item() - mindet) < 1e-12 * abs(mindet)


def _ops(N, E, lam, seed=fem_synth.SEED_Q, jitter=0.1):
    v = _mesh(E, jitter=jitter)
    q = fem_synth.field(seed, E, (N + 1) ** 3)
    return v, q


@pytest.mark.parametrize("N", range(1, 16))
def test_bp1_parity(bases, N):
    fem = _fem()
    v, q = _ops(N, E_RAGGED, 0.0)
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    ref = oracle.bp1(N, wJ, q)
    got = fem.fem_bp1_apply(bases[N], _dev(wJ), _dev(q)).cpu().numpy()
    assert _rel(got, ref) < TOL


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.37])
@pytest.mark.parametrize("N", range(1, 16))
def test_bp35_parity(bases, N, lam):
    fem = _fem()
    v, q = _ops(N, E_RAGGED, lam)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    ref = oracle.bp35(N, G, lam, q)
    got = fem.fem_bp35_apply(bases[N], _dev(G), lam, _dev(q)).cpu().numpy()
    assert _rel(got, ref) < TOL


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.37])
@pytest.mark.parametrize("N", range(1, 16))
def test_bp30_parity(bases, N, lam):
    fem = _fem()
    v, q = _ops(N, E_RAGGED, lam)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    ref = oracle.bp30(N, G, lam, q)
    got = fem.fem_bp30_apply(bases[N], _dev(G), lam, _dev(q)).cpu().numpy()
    assert _rel(got, ref) < TOL


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.37])
@pytest.mark.parametrize("N", range(1, 16))
def test_bp1_bp30_fused(bases, N, lam):
    """BP1.0 and BP3.0 of one field in one pass: bit for bit the separate
    kernels' outputs (BP1.0 with the seventh BP3.0 plane as wJ), and the
    oracle's to 1e-12; Mq, Aq and q must be distinct buffers."""
    fem, torch = _fem(), _torch()
    v, q = _ops(N, E_RAGGED, lam)
    b = bases[N]
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    Gd, qd = _dev(G), _dev(q)
    Mq, Aq = fem.fem_bp1_bp30_apply(b, Gd, lam, qd)
    wJ = Gd[:, 6, :].contiguous()
    assert torch.equal(Mq, fem.fem_bp1_apply(b, wJ, qd))
    assert torch.equal(Aq, fem.fem_bp30_apply(b, Gd, lam, qd))
    assert _rel(Mq.cpu().numpy(), oracle.bp1(N, np.ascontiguousarray(G[:, 6, :]), q)) < TOL
    assert _rel(Aq.cpu().numpy(), oracle.bp30(N, G, lam, q)) < TOL
    with pytest.raises(fem.FemError):
        fem.fem_bp1_bp30_apply(b, Gd, lam, qd, out_m=Aq, out_a=Aq)


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.37])
@pytest.mark.parametrize("N", range(1, 16))
def test_bp30_point_layout_parity(bases, N, lam):
    """The point-per-thread layout of BP3.0 against the oracle, with a
    ragged element count (one element per block; above m^3 = 1024 points a
    thread takes several)."""
    fem = _fem()
    v, q = _ops(N, E_RAGGED, lam)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    ref = oracle.bp30(N, G, lam, q)
    got = fem.fem_bp30_apply_layout(bases[N], _dev(G), lam, _dev(q), fem.FEM_LAYOUT_POINTS).cpu().numpy()
    assert _rel(got, ref) < TOL


@pytest.mark.parametrize("lam", [0.0, 1.0, 0.37])
@pytest.mark.parametrize("N", range(1, 16))
def test_bp35_point_layout_parity(bases, N, lam):
    """The point-per-thread layout of BP3.5 (Algorithm 7) against the oracle,
    with a ragged element count (one element per block; above n^3 = 1024
    nodes a thread takes several)."""
    fem = _fem()
    v, q = _ops(N, E_RAGGED, lam)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    ref = oracle.bp35(N, G, lam, q)
    got = fem.fem_bp35_apply_layout(bases[N], _dev(G), lam, _dev(q), fem.FEM_LAYOUT_POINTS).cpu().numpy()
    assert _rel(got, ref) < TOL
    lines = fem.fem_bp35_apply_layout(bases[N], _dev(G), lam, _dev(q), fem.FEM_LAYOUT_LINES).cpu().numpy()
    assert np.array_equal(lines, fem.fem_bp35_apply(bases[N], _dev(G), lam, _dev(q)).cpu().numpy())


@pytest.mark.parametrize("N", [1, 2, 7, 15])
def test_chain_from_vertices(bases, N):
    """Vertices -> device geometric factors -> device operators, against the
    oracle's own chain (no value crosses from one side to the other)."""
    fem = _fem()
    E = 19
    v, q = _ops(N, E, 1.0, seed=7, jitter=0.2)
    vd, qd = _dev(v), _dev(q)
    b = bases[N]
    for kind, apply_gpu, apply_or in (
        (1, lambda g: fem.fem_bp1_apply(b, g, qd), lambda g: oracle.bp1(N, g, q)),
        (2, lambda g: fem.fem_bp35_apply(b, g, 1.3, qd), lambda g: oracle.bp35(N, g, 1.3, q)),
        (3, lambda g: fem.fem_bp30_apply(b, g, 1.3, qd), lambda g: oracle.bp30(N, g, 1.3, q)),
    ):
        got = apply_gpu(fem.fem_mesh_geofacs(b, kind, vd)).cpu().numpy()
        ref = apply_or(oracle.geofacs(N, kind, v)[0])
        assert _rel(got, ref) < TOL


@pytest.mark.parametrize("N", [1, 7, 15])
def test_single_element_and_empty(bases, N):
    fem, torch = _fem(), _torch()
    b = bases[N]
    v, q = _ops(N, 1, 1.0)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    got = fem.fem_bp30_apply(b, _dev(G), 1.0, _dev(q)).cpu().numpy()
    assert _rel(got, oracle.bp30(N, G, 1.0, q)) < TOL
    # E = 0: a valid no-op
    q0 = torch.empty((0, (N + 1) ** 3), dtype=torch.float64, device="cuda")
    for kind in (1, 2, 3):
        g0 = torch.empty(fem.geo_shape(b, kind, 0), dtype=torch.float64, device="cuda")
        fem.fem_mesh_geofacs(b, kind, torch.empty((0, 8, 3), dtype=torch.float64, device="cuda"), geo=g0)
    fem.fem_bp1_apply(b, torch.empty((0, (N + 2) ** 3), dtype=torch.float64, device="cuda"), q0)
    fem.fem_bp35_apply(b, torch.empty((0, 7, (N + 1) ** 3), dtype=torch.float64, device="cuda"), 1.0, q0)
    fem.fem_bp30_apply(b, torch.empty((0, 7, (N + 2) ** 3), dtype=torch.float64, device="cuda"), 1.0, q0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("N", [3, 8])
def test_every_output_written(bases, N):
    """Outputs pre-filled with NaN come back finite everywhere (every entry is
    written, none is read before it is written)."""
    fem, torch = _fem(), _torch()
    E = 53
    v, q = _ops(N, E, 1.0)
    b = bases[N]
    vd, qd = _dev(v), _dev(q)
    for kind in (1, 2, 3):
        g = torch.full(fem.geo_shape(b, kind, E), float("nan"), dtype=torch.float64, device="cuda")
        fem.fem_mesh_geofacs(b, kind, vd, geo=g)
        assert torch.isfinite(g).all()
        out = torch.full_like(qd, float("nan"))
        if kind == 1:
            fem.fem_bp1_apply(b, g, qd, out=out)
        elif kind == 2:
            fem.fem_bp35_apply(b, g, 1.0, qd, out=out)
        else:
            fem.fem_bp30_apply(b, g, 1.0, qd, out=out)
        assert torch.isfinite(out).all()


def test_side_stream_and_aliasing_rejected(bases):
    fem, torch = _fem(), _torch()
    N = 4
    b = bases[N]
    v, q = _ops(N, 10, 1.0)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    s = torch.cuda.Stream()
    Gd, qd = _dev(G), _dev(q)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out = fem.fem_bp35_apply(b, Gd, 1.0, qd, stream=s)
    s.synchronize()
    assert _rel(out.cpu().numpy(), oracle.bp35(N, G, 1.0, q)) < TOL
    with pytest.raises(fem.FemError):
        fem.fem_bp35_apply(b, Gd, 1.0, qd, out=qd)  # in place is rejected


def test_inverted_element_flagged(bases):
    fem, torch = _fem(), _torch()
    v = _mesh(4)
    v[2] = v[2][[1, 0, 3, 2, 5, 4, 7, 6]]  # mirror element 2 in r
    dmin = torch.zeros(4, dtype=torch.float64, device="cuda")
    fem.fem_mesh_geofacs(bases[3], 3, _dev(v), detJ_min=dmin)
    d = dmin.cpu().numpy()
    assert d[2] < 0 and np.all(d[[0, 1, 3]] > 0)


# --------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def big_mesh():
    return fem_synth.box_mesh(32)  # E = 32768 jittered hexes of the unit cube


@pytest.mark.parametrize("N", range(1, 16))
def test_full_size_sampled(bases, big_mesh, N):
    """The 32^3 mesh at every degree of the sweep (N = 7 is the step's), in
    the launch configuration bench.py times; the oracle recomputes 48
    sampled elements (the operator is block diagonal, so each element's
    output depends on that element's data alone)."""
    fem, torch = _fem(), _torch()
    b = bases[N]
    v = big_mesh
    E = v.shape[0]
    q = fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)
    vd, qd = _dev(v), _dev(q)
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([rng.choice(E, 46, replace=False), [0, E - 1]]))
    vs, qs = v[pick], q[pick]
    for kind in (1, 2, 3):
        g = fem.fem_mesh_geofacs(b, kind, vd)
        if kind == 1:
            out = fem.fem_bp1_apply(b, g, qd)
            ref = oracle.bp1(N, oracle.geofacs(N, kind, vs)[0], qs)
        elif kind == 2:
            out = fem.fem_bp35_apply(b, g, 1.0, qd)
            ref = oracle.bp35(N, oracle.geofacs(N, kind, vs)[0], 1.0, qs)
        else:
            out = fem.fem_bp30_apply(b, g, 1.0, qd)
            ref = oracle.bp30(N, oracle.geofacs(N, kind, vs)[0], 1.0, qs)
        got = out[torch.from_numpy(pick).cuda()].cpu().numpy()
        assert _rel(got, ref) < TOL
        del g, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N", [1, 3, 4, 7, 9, 10, 15])
def test_full_size_sampled_reduced_precision(bases, big_mesh, N):
    """The FP32 and FP16-factor BP3.5 and BP3.0 operators of the sweep on the
    32^3 mesh (stream kernels up to N = 9, block kernels above), 48 sampled
    elements against the oracle applied to the same rounded factors and
    field: the difference is FP32 arithmetic only."""
    fem, torch = _fem(), _torch()
    b = bases[N]
    vd = _dev(big_mesh)
    E = vd.shape[0]
    q32 = _dev(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).float()
    rng = np.random.default_rng(1)
    pick = np.unique(np.concatenate([rng.choice(E, 46, replace=False), [0, E - 1]]))
    tp = torch.from_numpy(pick).cuda()
    qs = q32[tp].cpu().numpy().astype(np.float64)
    for kind, f32, f16, ref_op in ((2, fem.fem_bp35_apply_f32, fem.fem_bp35_apply_f16g, oracle.bp35),
                                   (3, fem.fem_bp30_apply_f32, fem.fem_bp30_apply_f16g, oracle.bp30)):
        g = fem.fem_mesh_geofacs(b, kind, vd)
        g32 = g.float()
        got = f32(b, g32, 1.0, q32)[tp].cpu().numpy().astype(np.float64)
        ref = ref_op(N, g32[tp].cpu().numpy().astype(np.float64), 1.0, qs)
        assert _rel(got, ref) < 2e-6 * (N + 2), ("f32", kind)
        del g32
        ex = int(np.frexp(g.abs().max().item())[1])
        gi = torch.tensor([2.0 ** (ex - 14)], dtype=torch.float64, device="cuda")
        g16 = (g * 2.0 ** (14 - ex)).half()
        del g
        got = f16(b, g16, gi, 1.0, q32)[tp].cpu().numpy().astype(np.float64)
        ref = ref_op(N, g16[tp].cpu().numpy().astype(np.float64) * 2.0 ** (ex - 14), 1.0, qs)
        assert _rel(got, ref) < 2e-6 * (N + 2), ("f16", kind)
        del g16
        torch.cuda.empty_cache()
    assert fem.fem_wait_timeouts() == 0


def test_factor_arrays_beyond_2_31_entries(bases):
    """N = 15 on an 80000-element mesh (50 x 40 x 40): the BP3.5 and BP3.0
    factor arrays hold 2.29e9 and 2.75e9 entries, beyond 32-bit indexing.
    Elements near the end, whose factors lie past entry 2^31, and a few at
    the start are checked against the oracle in FP64, FP32 and FP16 factors."""
    fem, torch = _fem(), _torch()
    N = 15
    b = bases[N]
    v = fem_synth.box_mesh(50, 40, 40)
    E = v.shape[0]
    assert E == 80000 and E * 7 * (N + 1) ** 3 > 2 ** 31
    vd = _dev(v)
    q = _dev(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3))
    pick = np.array([0, 1, 17, E - 4000, E - 777, E - 2, E - 1])
    tp = torch.from_numpy(pick).cuda()
    qs = q[tp].cpu().numpy()
    q32 = q.float()
    qs32 = q32[tp].cpu().numpy().astype(np.float64)
    for kind, f64, f32, f16, ref_op in ((2, fem.fem_bp35_apply, fem.fem_bp35_apply_f32, fem.fem_bp35_apply_f16g,
                                         oracle.bp35),
                                        (3, fem.fem_bp30_apply, fem.fem_bp30_apply_f32, fem.fem_bp30_apply_f16g,
                                         oracle.bp30)):
        g = fem.fem_mesh_geofacs(b, kind, vd)
        gs_oracle, _ = oracle.geofacs(N, kind, v[pick])
        assert _rel(g[tp].cpu().numpy(), gs_oracle) < TOL
        assert _rel(f64(b, g, 1.0, q)[tp].cpu().numpy(), ref_op(N, gs_oracle, 1.0, qs)) < TOL
        g32 = g.float()
        got = f32(b, g32, 1.0, q32)[tp].cpu().numpy().astype(np.float64)
        assert _rel(got, ref_op(N, g32[tp].cpu().numpy().astype(np.float64), 1.0, qs32)) < 2e-6 * (N + 2)
        del g32
        ex = int(np.frexp(g.abs().max().item())[1])
        gi = torch.tensor([2.0 ** (ex - 14)], dtype=torch.float64, device="cuda")
        g16 = (g * 2.0 ** (14 - ex)).half()
        del g
        got = f16(b, g16, gi, 1.0, q32)[tp].cpu().numpy().astype(np.float64)
        gr = g16[tp].cpu().numpy().astype(np.float64) * 2.0 ** (ex - 14)
        assert _rel(got, ref_op(N, gr, 1.0, qs32)) < 2e-6 * (N + 2)
        del g16
        torch.cuda.empty_cache()


def test_full_size_invariants(bases, big_mesh):
    """Properties that hold at any size, checked on the whole 32^3 mesh:
    1^T M 1 = 1 (unit-cube volume) and A 1 = 0 for lambda = 0."""
    fem, torch = _fem(), _torch()
    vd = _dev(big_mesh)
    for N in (3, 7):
        b = bases[N]
        one = torch.ones((vd.shape[0], (N + 1) ** 3), dtype=torch.float64, device="cuda")
        wJ = fem.fem_mesh_geofacs(b, 1, vd)
        assert abs(fem.fem_bp1_apply(b, wJ, one).sum().item() - 1.0) < 1e-12
        G30 = fem.fem_mesh_geofacs(b, 3, vd)
        ref = fem.fem_bp30_apply(b, G30, 0.0, torch.rand_like(one)).abs().max().item()
        assert fem.fem_bp30_apply(b, G30, 0.0, one).abs().max().item() < 1e-12 * ref
        del G30
        G35 = fem.fem_mesh_geofacs(b, 2, vd)
        ref = fem.fem_bp35_apply(b, G35, 0.0, torch.rand_like(one)).abs().max().item()
        assert fem.fem_bp35_apply(b, G35, 0.0, one).abs().max().item() < 1e-12 * ref


def test_small_bp1_config_full_oracle(bases):
    """BP1.0, N = 3, E = 512 (8^3 jittered cube): every element against the oracle."""
    fem = _fem()
    N = 3
    v = fem_synth.box_mesh(8)
    q = fem_synth.field(fem_synth.SEED_Q, v.shape[0], (N + 1) ** 3)
    wJ_ref, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    ref = oracle.bp1(N, wJ_ref, q)
    b = bases[N]
    got = fem.fem_bp1_apply(b, fem.fem_mesh_geofacs(b, 1, _dev(v)), _dev(q)).cpu().numpy()
    assert _rel(got, ref) < TOL


@pytest.mark.parametrize("dtype,planes,n", [("float64", 1, 2), ("float64", 8, 4096 * 3 + 2),
                                            ("float64", 25, 1 << 16), ("float32", 3, 4),
                                            ("float32", 9, 100_004), ("float32", 32, 1 << 15)])
def test_stream_sum_calibration_kernel(dtype, planes, n):
    """The roofline calibration stream sums its planes in plane order: bit
    for bit the sequential sum on the host."""
    import torch
    fem = _fem()
    src = fem_synth.field(31, planes, n).astype(dtype)
    ref = src[0].copy()
    for p in range(1, planes):
        ref = (ref + src[p]).astype(dtype)
    got = fem.fem_stream_sum(torch.from_numpy(src).to("cuda")).cpu().numpy()
    assert got.dtype == np.dtype(dtype)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("N", [1, 4, 7, 15])
def test_geofacs_set_equals_single_kind_calls(N):
    """All three factor sets in one call (wJ from the BP3.0 kernel) are the
    single-kind results bit for bit, and every subset works."""
    import torch
    fem = _fem()
    v = fem_synth.box_mesh(3)
    E = v.shape[0]
    b = fem.fem_basis_setup(N)
    vd = torch.from_numpy(v).to("cuda")
    ref = [fem.fem_mesh_geofacs(b, k, vd) for k in (1, 2, 3)]
    outs = [torch.full(fem.geo_shape(b, k, E), float("nan"), dtype=torch.float64, device="cuda") for k in (1, 2, 3)]
    fem.fem_mesh_geofacs_set(b, vd, *outs)
    for got, want in zip(outs, ref):
        assert torch.equal(got, want)
    w1 = torch.zeros_like(outs[0])
    fem.fem_mesh_geofacs_set(b, vd, wJ=w1)
    assert torch.equal(w1, ref[0])
    g3 = torch.zeros_like(outs[2])
    fem.fem_mesh_geofacs_set(b, vd, G30=g3)
    assert torch.equal(g3, ref[2])
    wJo, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    assert _rel(outs[0].cpu().numpy(), wJo) < 1e-13


def test_fma_probe_runs_and_is_deterministic():
    """The FP64 issue-rate probe: one double per thread, the same bits on a
    second launch, and the closed form of the chain x <- x b + c for the
    first chain of thread 0 of block 0."""
    import torch
    fem = _fem()
    out, flops = fem.fem_fma_probe(50)
    a = out.clone()
    fem.fem_fma_probe(50, out=out)
    torch.cuda.synchronize()
    assert torch.equal(a, out) and flops == 2 * 8 * 50 * out.numel()
    b, c = 0.999999, 1e-6
    xs = [i * 1e-3 for i in range(8)]
    for _ in range(50):
        xs = [x * b + c for x in xs]
    assert abs(out[0].item() - sum(xs)) <= 1e-12


@pytest.mark.parametrize("N", [1, 4, 9, 15])
@pytest.mark.parametrize("E", [1, 7, 64])
def test_affine_mesh_parity_from_vertices(bases, N, E):
    """Undistorted (affine, axis-aligned) elements, from the vertices through
    the factor-set call to the three operators, against the oracle at
    several element counts."""
    fem, torch = _fem(), _torch()
    v = _mesh(E, jitter=0.0)
    q = fem_synth.field(17, E, (N + 1) ** 3)
    b = bases[N]
    vd = _dev(v)
    wJ = torch.empty(fem.geo_shape(b, 1, E), dtype=torch.float64, device="cuda")
    G35 = torch.empty(fem.geo_shape(b, 2, E), dtype=torch.float64, device="cuda")
    G30 = torch.empty(fem.geo_shape(b, 3, E), dtype=torch.float64, device="cuda")
    fem.fem_mesh_geofacs_set(b, vd, wJ=wJ, G35=G35, G30=G30)
    qd = _dev(q)
    wJo, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    G35o, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    G30o, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    assert _rel(fem.fem_bp1_apply(b, wJ, qd).cpu().numpy(), oracle.bp1(N, wJo, q)) < TOL
    assert _rel(fem.fem_bp35_apply(b, G35, 1.0, qd).cpu().numpy(), oracle.bp35(N, G35o, 1.0, q)) < TOL
    assert _rel(fem.fem_bp30_apply(b, G30, 1.0, qd).cpu().numpy(), oracle.bp30(N, G30o, 1.0, q)) < TOL


@pytest.mark.parametrize("N", [3, 7])
def test_512_element_mesh_all_operators(bases, N):
    """The 8^3 mesh of the small configuration (512 jittered elements) for all
    three operators, element by element against the oracle."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(8)
    E = v.shape[0]
    q = fem_synth.field(2, E, (N + 1) ** 3)
    b = bases[N]
    vd, qd = _dev(v), _dev(q)
    for kind, apply_gpu, apply_o in ((oracle.KIND_BP1, lambda g: fem.fem_bp1_apply(b, g, qd),
                                      lambda g: oracle.bp1(N, g, q)),
                                     (oracle.KIND_BP35, lambda g: fem.fem_bp35_apply(b, g, 1.0, qd),
                                      lambda g: oracle.bp35(N, g, 1.0, q)),
                                     (oracle.KIND_BP30, lambda g: fem.fem_bp30_apply(b, g, 1.0, qd),
                                      lambda g: oracle.bp30(N, g, 1.0, q))):
        go, _ = oracle.geofacs(N, kind, v)
        gd = fem.fem_mesh_geofacs(b, kind, vd)
        assert _rel(gd.cpu().numpy(), go) < TOL
        assert _rel(apply_gpu(gd).cpu().numpy(), apply_o(go)) < TOL

"""GPU checks of the precision row: the FP32 BP3.5 matvec, the Jacobi
diagonal, the deterministic dot product, and the FP64 and mixed-precision
(FP32 inner solves inside FP64 defect correction) Jacobi-PCG solvers, against
the FP64 oracle and the manufactured discrete solution."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def _fem():
    import paper_1711_00903_gb300 as fem
    return fem


def _torch():
    import torch
    return torch


def _dev(a):
    return _torch().from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(got, ref):
    return np.abs(np.asarray(got) - ref).max() / np.abs(ref).max()


def _manufactured(N, nx, lam=1.0):
    """b = A_oracle u_I, u_I = sin(pi x) sin(pi y) sin(pi z) at the GLL nodes."""
    v = fem_synth.box_mesh(nx)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    X = oracle.gll_node_coordinates(N, v)
    u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    b = oracle.bp35(N, G, lam, u)
    return v, G, u, b


@pytest.mark.parametrize("N", [1, 3, 7, 15])
def test_jacobi_diagonal(N):
    fem = _fem()
    v = fem_synth.box_mesh(3)[:23]
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    b = fem.fem_basis_setup(N)
    got = fem.fem_bp35_jacobi(b, _dev(G), 1.0).cpu().numpy()
    ref = 1.0 / oracle.bp35_diag(N, G, 1.0)
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9, 11, 13, 15])
def test_bp35_f32_matches_fp64_operator(N):
    """FP32 matvec against the FP64 oracle applied to the same FP32-rounded
    inputs: the difference is FP32 rounding of the arithmetic only."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(3)[:19]
    E = v.shape[0]
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    q = fem_synth.field(2, E, (N + 1) ** 3)
    G32, q32 = G.astype(np.float32), q.astype(np.float32)
    ref = oracle.bp35(N, G32.astype(np.float64), 1.0, q32.astype(np.float64))
    b = fem.fem_basis_setup(N)
    got = fem.fem_bp35_apply_f32(b, _dev(G32), 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
    assert _rel(got, ref) < 2e-6 * (N + 1)


@pytest.mark.parametrize("N", [1, 2, 5, 7, 11, 15])
def test_bp30_f32_matches_fp64_operator(N):
    """FP32 BP3.0 matvec against the FP64 oracle on the same FP32-rounded
    inputs; the bound grows with the length of the contraction chain."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(3)[:19]
    E = v.shape[0]
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    q = fem_synth.field(2, E, (N + 1) ** 3)
    G32, q32 = G.astype(np.float32), q.astype(np.float32)
    ref = oracle.bp30(N, G32.astype(np.float64), 1.0, q32.astype(np.float64))
    b = fem.fem_basis_setup(N)
    got = fem.fem_bp30_apply_f32(b, _dev(G32), 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
    assert _rel(got, ref) < 2e-6 * (N + 2)


@pytest.mark.parametrize("op,N", [("bp35", 7), ("bp35", 5), ("bp35", 4), ("bp35", 8), ("bp35", 10), ("bp35", 12),
                                  ("bp35", 15), ("bp30", 7), ("bp30", 4), ("bp30", 9)])
def test_stream_kernels_many_groups_per_block(op, N):
    """The FP32 and FP16-factor operators on 1001 elements: for BP3.5 the TMA
    stream kernels with several element groups per persistent block (stages
    reused; above N = 9 the kernel with one factor stage, whose next copy
    starts in the middle of the element), and at even N element ranges off
    16-byte boundaries (range copies, with the plain-load tail at the end of
    the arrays); for BP3.0 the block kernels.  Against the oracle on the same
    rounded inputs."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(11, 10, 10)[:1001]
    E = v.shape[0]
    kind = oracle.KIND_BP35 if op == "bp35" else oracle.KIND_BP30
    G, _ = oracle.geofacs(N, kind, v)
    q32 = fem_synth.field(9, E, (N + 1) ** 3).astype(np.float32)
    b = fem.fem_basis_setup(N)
    apply = oracle.bp35 if op == "bp35" else oracle.bp30
    ref32 = apply(N, G.astype(np.float32).astype(np.float64), 1.0, q32.astype(np.float64))
    f32 = fem.fem_bp35_apply_f32 if op == "bp35" else fem.fem_bp30_apply_f32
    got = f32(b, _dev(G.astype(np.float32)), 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
    assert _rel(got, ref32) < 2e-6 * (N + 2)
    G16, ginv = _f16_factors(G)
    ref16 = apply(N, G16.astype(np.float64) * ginv, 1.0, q32.astype(np.float64))
    f16 = fem.fem_bp35_apply_f16g if op == "bp35" else fem.fem_bp30_apply_f16g
    gi = torch.tensor([ginv], dtype=torch.float64, device="cuda")
    got = f16(b, torch.from_numpy(G16).to("cuda"), gi, 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
    assert _rel(got, ref16) < 2e-6 * (N + 2)
    assert fem.fem_wait_timeouts() == 0


def test_stream_f32_operator_ragged_groups_and_no_wait_timeouts():
    """The FP32 BP3.5 kernels that stage the factors with TMA bulk copies
    (two stages up to N = 9, one factor stage above): a single element,
    element counts that leave the last group partly filled, results equal
    to the oracle's on the same FP32 inputs, and no bounded wait gave up."""
    fem, torch = _fem(), _torch()
    fem.fem_wait_timeouts(reset=True)
    for N, E in ((7, 1), (7, 37), (3, 33), (4, 7), (8, 5), (10, 1), (11, 3), (14, 2), (15, 5)):
        v = fem_synth.box_mesh(4)[:E]
        G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
        q = fem_synth.field(3, E, (N + 1) ** 3)
        G32, q32 = G.astype(np.float32), q.astype(np.float32)
        ref = oracle.bp35(N, G32.astype(np.float64), 1.0, q32.astype(np.float64))
        b = fem.fem_basis_setup(N)
        got = fem.fem_bp35_apply_f32(b, _dev(G32), 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
        assert _rel(got, ref) < 2e-6 * (N + 1)
    assert fem.fem_wait_timeouts() == 0


def _f16_factors(G):
    """binary16 factors scaled by 2^(14 - e), max|G| < 2^e, as the solver
    scales them, and the inverse scale."""
    e = int(np.frexp(np.abs(G).max())[1])
    s = 2.0 ** (14 - e)
    G16 = (G * s).astype(np.float16)
    return G16, 1.0 / s


@pytest.mark.parametrize("op", ["bp35", "bp30"])
@pytest.mark.parametrize("N", [1, 2, 3, 6, 7, 9, 12, 15])
def test_f16_factor_operators(op, N):
    """Half-precision-factor operators against the FP64 oracle applied to the
    same rounded factors (unscaled) and the same FP32-rounded field: the
    difference is FP32 arithmetic only.  Odd N up to 9 exercise the BP3.5
    stream kernel with FP16 stages, the others the block kernels."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(3)[:23]
    E = v.shape[0]
    kind = oracle.KIND_BP35 if op == "bp35" else oracle.KIND_BP30
    G, _ = oracle.geofacs(N, kind, v)
    G16, ginv = _f16_factors(G)
    q32 = fem_synth.field(7, E, (N + 1) ** 3).astype(np.float32)
    Gr = G16.astype(np.float64) * ginv
    ref = (oracle.bp35 if op == "bp35" else oracle.bp30)(N, Gr, 1.0, q32.astype(np.float64))
    b = fem.fem_basis_setup(N)
    gi = torch.tensor([ginv], dtype=torch.float64, device="cuda")
    fn = fem.fem_bp35_apply_f16g if op == "bp35" else fem.fem_bp30_apply_f16g
    got = fn(b, torch.from_numpy(G16).to("cuda"), gi, 1.0, _dev(q32)).cpu().numpy().astype(np.float64)
    assert _rel(got, ref) < 2e-6 * (N + 2)
    # the rounded factors are within binary16 precision of the FP64 ones
    assert np.abs(Gr - G).max() <= 2.0 ** -11 * np.abs(G).max()
    assert fem.fem_wait_timeouts() == 0


@pytest.mark.parametrize("op", ["bp35", "bp30"])
@pytest.mark.parametrize("N", [2, 7])
def test_apply_ex_selects_the_precision_entry_points(op, N):
    """The run-time-precision entry points give, bit for bit, the results of
    the entry point of each precision, and the FP64 one matches the oracle."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(3)[:23]
    E = v.shape[0]
    kind = oracle.KIND_BP35 if op == "bp35" else oracle.KIND_BP30
    G, _ = oracle.geofacs(N, kind, v)
    q = fem_synth.field(5, E, (N + 1) ** 3)
    b = fem.fem_basis_setup(N)
    ex = fem.fem_bp35_apply_ex if op == "bp35" else fem.fem_bp30_apply_ex
    f64 = fem.fem_bp35_apply if op == "bp35" else fem.fem_bp30_apply
    f32 = fem.fem_bp35_apply_f32 if op == "bp35" else fem.fem_bp30_apply_f32
    f16 = fem.fem_bp35_apply_f16g if op == "bp35" else fem.fem_bp30_apply_f16g
    Gd, qd = _dev(G), _dev(q)
    got = ex(b, fem.FEM_PREC_F64, Gd, 1.0, qd)
    assert torch.equal(got, f64(b, Gd, 1.0, qd))
    assert _rel(got.cpu().numpy(), (oracle.bp35 if op == "bp35" else oracle.bp30)(N, G, 1.0, q)) <= 1e-12
    G32, q32 = Gd.float(), qd.float()
    assert torch.equal(ex(b, fem.FEM_PREC_F32, G32, 1.0, q32), f32(b, G32, 1.0, q32))
    G16, ginv = _f16_factors(G)
    G16d, gi = torch.from_numpy(G16).to("cuda"), torch.tensor([ginv], dtype=torch.float64, device="cuda")
    assert torch.equal(ex(b, fem.FEM_PREC_F16G, G16d, 1.0, q32, ginv=gi), f16(b, G16d, gi, 1.0, q32))
    tc = fem.fem_bp30_apply_tc if op == "bp30" else fem.fem_bp35_apply_tc
    assert torch.equal(ex(b, fem.FEM_PREC_F16TC, G32, 1.0, q32), tc(b, G32, 1.0, q32))
    with pytest.raises(ValueError):
        ex(b, 4, Gd, 1.0, qd)
    with pytest.raises(TypeError):
        ex(b, fem.FEM_PREC_F32, Gd, 1.0, qd)  # float64 tensors for the FP32 path


def test_dot_deterministic_and_exact():
    fem, torch = _fem(), _torch()
    x = fem_synth.field(11, 1, 3_000_001)[0]
    y = fem_synth.field(12, 1, 3_000_001)[0]
    xd, yd = _dev(x), _dev(y)
    r1 = fem.fem_dot(xd, yd).item()
    r2 = fem.fem_dot(xd, yd).item()
    assert r1 == r2
    ref = float(np.dot(x, y))
    assert abs(r1 - ref) <= 1e-12 * np.abs(x * y).sum()
    assert fem.fem_dot(xd[:0], yd[:0]).item() == 0.0


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["fp64", "mixed", "mixed16"])
@pytest.mark.parametrize("N", [2, 4, 7])
def test_pcg_manufactured(N, mode):
    fem = _fem()
    v, G, u, b = _manufactured(N, 4)
    basis = fem.fem_basis_setup(N)
    Gd = _dev(G)
    s = fem.fem_pcg_create(basis, Gd, 1.0, mode)
    x, info, code = s.solve(_dev(b), tol=1e-12 if mode == 0 else 1e-11)
    x = x.cpu().numpy()
    assert code == 0
    assert info["relres"] <= (1e-12 if mode == 0 else 1e-11) * 1.0001
    # true residual recomputed by the oracle
    tr = np.linalg.norm(b - oracle.bp35(N, G, 1.0, x)) / np.linalg.norm(b)
    assert tr <= 2e-11
    lim = 1e-8 if mode == 0 else 1e-7
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= lim
    # against the oracle's own PCG solve
    xo, it_o, _ = oracle.pcg_bp35(N, G, 1.0, b, tol=1e-12)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= lim
    if mode == 0:
        assert abs(info["iters"] - it_o) <= 2
    else:
        assert info["outer"] >= 2


def test_pcg_result_independent_of_check_period_and_repeatable():
    fem = _fem()
    N = 3
    v, G, u, b = _manufactured(N, 3)
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, 0)
    bd = _dev(b)
    x1, i1, _ = s.solve(bd, tol=1e-10, check_every=1)
    x2, i2, _ = s.solve(bd, tol=1e-10, check_every=7)
    x3, i3, _ = s.solve(bd, tol=1e-10, check_every=7)
    assert i1["iters"] == i2["iters"] == i3["iters"]
    assert bool((x1 == x2).all()) and bool((x2 == x3).all())


def test_pcg_edge_cases():
    fem, torch = _fem(), _torch()
    N = 2
    v, G, u, b = _manufactured(N, 2)
    basis = fem.fem_basis_setup(N)
    Gd = _dev(G)
    with pytest.raises(fem.FemError):
        fem.fem_pcg_create(basis, Gd, -1.0, 0)
    with pytest.raises(fem.FemError):
        fem.fem_pcg_create(basis, Gd, 1.0, 7)
    for mode in (0, 1):
        s = fem.fem_pcg_create(basis, Gd, 1.0, mode)
        zero = torch.zeros((v.shape[0], 27), dtype=torch.float64, device="cuda")
        x, info, code = s.solve(zero, x=torch.ones_like(zero))
        assert code == 0 and float(x.abs().max()) == 0.0
        # iteration limit reached: FEM_ENOCONV, x holds the last iterate
        x, info, code = s.solve(_dev(b), tol=1e-14, maxit=2, inner_maxit=1, raise_on_error=False)
        assert code == fem.FEM_ENOCONV
        assert np.all(np.isfinite(x.cpu().numpy()))


def _full_size_manufactured(fem, N):
    """The 32^3 mesh (E = 32768) with its BP3.5 factors, u_I and b = A u_I,
    on the device."""
    v = fem_synth.box_mesh(32)
    basis = fem.fem_basis_setup(N)
    vd = _dev(v)
    G = fem.fem_mesh_geofacs(basis, fem.FEM_GEO_BP35, vd)
    X = oracle.gll_node_coordinates(N, v[:64])  # spot check of the coordinates below
    # u_I on the device from the same trilinear map (oracle coordinates for all
    # elements would take long; the map is evaluated by numpy here)
    r, _ = oracle.gll(N)
    n = N + 1
    R, S, T = np.meshgrid(r, r, r, indexing="ij")  # (i, j, k) grids
    R, S, T = R.transpose(2, 1, 0).reshape(-1), S.transpose(2, 1, 0).reshape(-1), T.transpose(2, 1, 0).reshape(-1)
    phi = np.stack([((1 + (1 if c & 1 else -1) * R) * (1 + (1 if c & 2 else -1) * S) *
                     (1 + (1 if c & 4 else -1) * T)) / 8 for c in range(8)], axis=1)  # (n^3, 8)
    Xall = np.einsum("pc,ecd->epd", phi, v)
    np.testing.assert_allclose(Xall[:64], X, rtol=0, atol=1e-14)
    u = np.sin(np.pi * Xall[..., 0]) * np.sin(np.pi * Xall[..., 1]) * np.sin(np.pi * Xall[..., 2])
    ud = _dev(u)
    bd = fem.fem_bp35_apply(basis, G, 1.0, ud)
    return basis, G, ud, bd


def test_full_size_mixed_solve_config():
    """N = 7 on the 32^3 mesh (E = 32768), manufactured right-hand side:
    the mixed solve reaches the FP64 tolerance and the discrete solution."""
    fem, torch = _fem(), _torch()
    basis, G, ud, bd = _full_size_manufactured(fem, 7)
    s = fem.fem_pcg_create(basis, G, 1.0, fem.FEM_PCG_MIXED)
    x, info, code = s.solve(bd, tol=1e-10)
    assert code == 0 and info["relres"] <= 1e-10
    err = (torch.linalg.norm(x - ud) / torch.linalg.norm(ud)).item()
    assert err <= 1e-7
    s64 = fem.fem_pcg_create(basis, G, 1.0, fem.FEM_PCG_FP64)
    x64, info64, code64 = s64.solve(bd, tol=1e-10)
    assert code64 == 0
    assert (torch.linalg.norm(x - x64) / torch.linalg.norm(x64)).item() <= 1e-7


def test_full_size_tight_tolerance():
    """On the 32^3 mesh at N = 7 the FP64 recurrence's residual drifts below
    the true one near 1e-12: FEM_OK still means a true residual within tol
    (the solver restarts from the true residual), a tolerance below FP64's
    reach ends in FEM_ENOCONV with a finite iterate, and at tol 1e-13 the
    mixed solves agree with the FP64 solve, and with u_I, to 1e-10."""
    fem, torch = _fem(), _torch()
    basis, G, ud, bd = _full_size_manufactured(fem, 7)
    rel = lambda a, b: (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
    s64 = fem.fem_pcg_create(basis, G, 1.0, fem.FEM_PCG_FP64)
    x64, info, code = s64.solve(bd, tol=1e-12)
    assert code == 0 and info["relres"] <= 1e-12
    x64, info, code = s64.solve(bd, tol=1e-13, raise_on_error=False)
    if code == 0:
        assert info["relres"] <= 1e-13
    else:
        assert code == fem.FEM_ENOCONV and bool(torch.isfinite(x64).all())
    assert info["relres"] <= 1e-11 and rel(x64, ud) <= 1e-10
    x_ref = x64.clone()
    x, info, code = s64.solve(bd, tol=1e-16, maxit=3000, raise_on_error=False)
    assert code == fem.FEM_ENOCONV and bool(torch.isfinite(x).all()) and info["relres"] <= 1e-11
    for mode in (fem.FEM_PCG_MIXED, fem.FEM_PCG_MIXED16, fem.FEM_PCG_MIXED_TC):
        s = fem.fem_pcg_create(basis, G, 1.0, mode)
        x, info, code = s.solve(bd, tol=1e-13, inner_tol=1e-3)
        assert code == 0 and info["relres"] <= 1e-13
        assert rel(x, x_ref) <= 1e-10 and rel(x, ud) <= 1e-10
        s.free()


# ------------------------------------------------------------------ BP3.0

@pytest.mark.parametrize("N", [1, 3, 7, 10])
def test_bp30_jacobi_diagonal(N):
    fem = _fem()
    v = fem_synth.box_mesh(3)[:11]
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    b = fem.fem_basis_setup(N)
    got = fem.fem_bp30_jacobi(b, _dev(G), 1.0).cpu().numpy()
    ref = 1.0 / oracle.bp30_diag(N, G, 1.0)
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("mode", [0, 1, 2, 3], ids=["fp64", "mixed", "mixed16", "mixed_tc"])
@pytest.mark.parametrize("N", [2, 5])
def test_bp30_pcg_manufactured(N, mode):
    fem = _fem()
    v = fem_synth.box_mesh(3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    X = oracle.gll_node_coordinates(N, v)
    u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    b = oracle.bp30(N, G, 1.0, u)
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, mode, op=fem.FEM_OP_BP30)
    x, info, code = s.solve(_dev(b), tol=1e-12 if mode == 0 else 1e-11)
    x = x.cpu().numpy()
    assert code == 0
    tr = np.linalg.norm(b - oracle.bp30(N, G, 1.0, x)) / np.linalg.norm(b)
    assert tr <= 2e-11
    lim = 1e-8 if mode == 0 else 1e-7
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= lim
    xo, it_o, _ = oracle.pcg_bp30(N, G, 1.0, b, tol=1e-12)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= lim
    if mode == 0:
        assert abs(info["iters"] - it_o) <= 2


def test_bp30_f32_matvec_through_mixed_solver_components():
    """The FP32 BP3.0 operator agrees with the FP64 one to FP32 rounding
    (checked through a one-outer-step mixed solve's first residual drop)."""
    fem = _fem()
    N = 4
    v = fem_synth.box_mesh(2)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    b = fem_synth.field(5, v.shape[0], (N + 1) ** 3)
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, fem.FEM_PCG_MIXED, op=fem.FEM_OP_BP30)
    x, info, code = s.solve(_dev(b), tol=1e-9, inner_tol=1e-5)
    assert code == 0 and info["outer"] <= 4


def test_solve_on_a_side_stream_replays_graphs_with_the_same_bits():
    """On a created stream the solver replays captured CUDA graphs of its
    iteration chunks; the result equals the direct launches on the default
    stream bit for bit, also when the right-hand side buffer changes."""
    import torch
    fem = _fem()
    for op, kind, apply in ((fem.FEM_OP_BP35, oracle.KIND_BP35, oracle.bp35),
                            (fem.FEM_OP_BP30, oracle.KIND_BP30, oracle.bp30)):
        N = 3
        v = fem_synth.box_mesh(3)
        G, _ = oracle.geofacs(N, kind, v)
        b1 = _dev(fem_synth.field(41, v.shape[0], 64))
        b2 = _dev(fem_synth.field(42, v.shape[0], 64))
        basis = fem.fem_basis_setup(N)
        for mode in (0, 1):
            s = fem.fem_pcg_create(basis, _dev(G), 1.0, mode, op=op)
            ref1, i1, _ = s.solve(b1, tol=1e-10)
            ref2, i2, _ = s.solve(b2, tol=1e-10)
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                x1, j1, _ = s.solve(b1, tol=1e-10, stream=st)
                x1b, j1b, _ = s.solve(b1, x=torch.zeros_like(b1), tol=1e-10, stream=st)
                x2, j2, _ = s.solve(b2, tol=1e-10, stream=st)
            st.synchronize()
            assert torch.equal(ref1, x1) and torch.equal(ref1, x1b) and torch.equal(ref2, x2)
            assert i1["iters"] == j1["iters"] and i2["iters"] == j2["iters"]


@pytest.mark.parametrize("N", [2, 4, 7])
def test_bp35_mixed_tc_manufactured(N):
    """BP3.5 defect correction with the tensor-core inner operator reaches
    the manufactured solution and the oracle's solve, as the FP32 mode does."""
    fem = _fem()
    v, G, u, b = _manufactured(N, 3)
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, fem.FEM_PCG_MIXED_TC)
    x, info, code = s.solve(_dev(b), tol=1e-11)
    x = x.cpu().numpy()
    assert code == 0 and info["relres"] <= 1e-11
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= 1e-7
    xo, _, _ = oracle.pcg_bp35(N, G, 1.0, b, tol=1e-12)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-7


def test_full_size_bp30_solves_all_modes():
    """The BP3.0 Helmholtz solve (lambda = 1) on the 32^3 jittered mesh at
    N = 7 with b = A u_I, in every mode to a 5e-13 relative residual (the
    FP64 BP3.0 residual stagnates near 2e-13 on this mesh): the FP32,
    FP16-factor and tensor-core defect-correction solves then reach the
    FP64 solution to 1e-10."""
    fem, torch = _fem(), _torch()
    N = 7
    v = fem_synth.box_mesh(32)
    basis = fem.fem_basis_setup(N)
    vd = _dev(v)
    G = fem.fem_mesh_geofacs(basis, fem.FEM_GEO_BP30, vd)
    X = oracle.gll_node_coordinates(N, v)
    u = _dev(np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2]))
    b = fem.fem_bp30_apply(basis, G, 1.0, u)
    xs = {}
    for mode in (fem.FEM_PCG_FP64, fem.FEM_PCG_MIXED, fem.FEM_PCG_MIXED16, fem.FEM_PCG_MIXED_TC):
        s = fem.fem_pcg_create(basis, G, 1.0, mode, op=fem.FEM_OP_BP30)
        x, info, code = s.solve(b, tol=5e-13, inner_tol=1e-3)
        assert code == 0, mode
        r = b - fem.fem_bp30_apply(basis, G, 1.0, x)
        assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() <= 1e-12, mode
        xs[mode] = x
        s.free()
    ref = xs[fem.FEM_PCG_FP64]
    for mode, x in xs.items():
        assert (torch.linalg.norm(x - ref) / torch.linalg.norm(ref)).item() <= 1e-10, mode


@pytest.mark.parametrize("N", [10, 13])
def test_high_degree_mixed_solves_match_fp64(N):
    """BP3.5 mixed solves above N = 9, whose inner operator is the stream
    kernel with one factor stage (FP32 and FP16 factors), reach the FP64
    solve of the same system."""
    fem, torch = _fem(), _torch()
    v = fem_synth.box_mesh(2)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    b = _dev(fem_synth.field(21, v.shape[0], (N + 1) ** 3))
    basis = fem.fem_basis_setup(N)
    xs = {}
    for mode in (fem.FEM_PCG_FP64, fem.FEM_PCG_MIXED, fem.FEM_PCG_MIXED16):
        s = fem.fem_pcg_create(basis, _dev(G), 1.0, mode)
        x, info, code = s.solve(b, tol=1e-11, inner_tol=1e-3)
        assert code == fem.FEM_OK and info["relres"] <= 1e-11
        xs[mode] = x
    for mode in (fem.FEM_PCG_MIXED, fem.FEM_PCG_MIXED16):
        d = (torch.linalg.norm(xs[mode] - xs[fem.FEM_PCG_FP64]) / torch.linalg.norm(xs[fem.FEM_PCG_FP64])).item()
        assert d <= 1e-8, mode
    assert fem.fem_wait_timeouts() == 0

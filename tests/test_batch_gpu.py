"""Batched BP3.5 / BP3.0 over many meshes of mixed degree in one persistent
launch: every element's result equals the per-mesh call bit for bit, and the
per-mesh calls equal the oracle; the autotuner and the CUDA-graph replay give
the same bits."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def _fem():
    import paper_1711_00903_gb300 as fem
    return fem


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _build(specs, bases):
    """(items, per-mesh reference outputs) for specs [(op, N, nx, ny, nz, seed)]."""
    import torch
    fem = _fem()
    items, refs = [], []
    for op, N, nx, ny, nz, seed in specs:
        b = bases[N]
        v = fem_synth.box_mesh(nx, ny, nz, jitter=0.1, seed=seed)
        E = v.shape[0]
        kind = fem.FEM_GEO_BP35 if op == fem.FEM_OP_BP35 else fem.FEM_GEO_BP30
        geo = fem.fem_mesh_geofacs(b, kind, _dev(v))
        q = _dev(fem_synth.field(seed + 1, E, (N + 1) ** 3))
        out = torch.full_like(q, float("nan"))
        lam = 0.5 + (seed % 3)
        ref = (fem.fem_bp35_apply if op == fem.FEM_OP_BP35 else fem.fem_bp30_apply)(b, geo, lam, q)
        items.append((op, b, geo, lam, q, out))
        refs.append((ref, v, lam))
    return items, refs


@pytest.fixture(scope="module")
def bases():
    fem = _fem()
    return {N: fem.fem_basis_setup(N) for N in range(1, 11)}


def test_mixed_batch_matches_per_mesh_calls_and_oracle(bases):
    import torch
    fem = _fem()
    specs = []
    for k, N in enumerate([1, 2, 3, 5, 7, 9, 10, 4]):
        specs.append((fem.FEM_OP_BP35, N, 2, 2, 1 + k % 3, 100 + k))
        specs.append((fem.FEM_OP_BP30, N, 1, 3, 2, 200 + k))
    specs.append((fem.FEM_OP_BP35, 6, 1, 1, 1, 300))  # a single element
    items, refs = _build(specs, bases)
    batch = fem.Batch(items)
    batch.apply()
    torch.cuda.synchronize()
    for (op, b, geo, lam, q, out), (ref, v, lam2), spec in zip(items, refs, specs):
        assert torch.equal(out, ref), spec
    # per-mesh calls against the oracle for a few of them
    for (op, b, geo, lam, q, out), (ref, v, _), spec in list(zip(items, refs, specs))[:6]:
        N = b.N
        if op == fem.FEM_OP_BP35:
            G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
            o = oracle.bp35(N, G, lam, q.cpu().numpy())
        else:
            G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
            o = oracle.bp30(N, G, lam, q.cpu().numpy())
        assert np.abs(out.cpu().numpy() - o).max() / np.abs(o).max() < 1e-12


def test_tuner_and_graph_replay_keep_the_bits(bases):
    import torch
    fem = _fem()
    specs = [(fem.FEM_OP_BP35 if k % 2 else fem.FEM_OP_BP30, 2 + k % 9, 3, 3, 2, 400 + k) for k in range(12)]
    items, refs = _build(specs, bases)
    batch = fem.Batch(items)
    results = batch.tune(reps=2)
    # the BP3.0 meshes of degree <= 8 and the BP3.5 meshes of degree <= 9
    # make both point layouts, alone and together, candidates too
    assert len(results) == 64 and all(r[4] > 0 for r in results)
    assert {r[3] for r in results} == {0, fem.FEM_BATCH_POINTS30, fem.FEM_BATCH_POINTS35,
                                       fem.FEM_BATCH_POINTS30 | fem.FEM_BATCH_POINTS35}
    cfg = batch.config
    assert cfg["ms"] == min(r[4] for r in results)
    if cfg["layout"] != fem.FEM_LAYOUT_LINES:  # compare with the lines layout below
        batch.config = {"threads": cfg["threads"], "group": cfg["group"], "order": cfg["order"]}
    for _, _, _, _, _, out in items:
        out.fill_(float("nan"))
    batch.graph_launch()
    batch.graph_launch()
    torch.cuda.synchronize()
    for (op, b, geo, lam, q, out), (ref, v, _) in zip(items, refs):
        assert torch.equal(out, ref)
    # every configuration gives the same bits
    for threads in (256, 512):
        for order in (0, 1):
            batch.config = {"threads": threads, "group": 3, "order": order}
            for _, _, _, _, _, out in items:
                out.zero_()
            batch.apply()
            torch.cuda.synchronize()
            for (op, b, geo, lam, q, out), (ref, v, _) in zip(items, refs):
                assert torch.equal(out, ref)


def test_point_layout_in_batch_matches_per_mesh_point_calls(bases):
    """BP3.0 tasks in the point layout: bit for bit the per-mesh call in the
    same layout, and within rounding of the lines layout and the oracle;
    BP3.5 tasks and BP3.0 above N = 8 keep the lines layout."""
    import torch
    fem = _fem()
    specs = [(fem.FEM_OP_BP30, N, 2, 1, 2, 500 + N) for N in (1, 3, 6, 8, 9)]
    specs.append((fem.FEM_OP_BP35, 4, 2, 2, 1, 600))
    items, refs = _build(specs, bases)
    batch = fem.Batch(items)
    batch.config = {"threads": 256, "group": 2, "order": 0, "layout": fem.FEM_LAYOUT_POINTS}
    batch.apply()
    torch.cuda.synchronize()
    for (op, b, geo, lam, q, out), (ref, v, _), spec in zip(items, refs, specs):
        if op == fem.FEM_OP_BP30 and b.N <= 8:
            pt = fem.fem_bp30_apply_layout(b, geo, lam, q, fem.FEM_LAYOUT_POINTS)
            assert torch.equal(out, pt), spec
            G, _ = oracle.geofacs(b.N, oracle.KIND_BP30, v)
            o = oracle.bp30(b.N, G, lam, q.cpu().numpy())
            assert np.abs(out.cpu().numpy() - o).max() / np.abs(o).max() < 1e-12, spec
            assert (out - ref).abs().max().item() / ref.abs().max().item() < 1e-12, spec
        else:
            assert torch.equal(out, ref), spec


@pytest.mark.parametrize("layout", [2, 3], ids=["points35", "points35+30"])
def test_bp35_point_layout_in_batch(bases, layout):
    """BP3.5 tasks up to N = 9 in the point layout (Algorithm 7): bit for bit
    the per-mesh call in the same layout and within rounding of the oracle;
    BP3.5 at N = 10 keeps the lines layout."""
    import torch
    fem = _fem()
    specs = [(fem.FEM_OP_BP35, N, 2, 1, 2, 700 + N) for N in (1, 2, 5, 9, 10)]
    specs.append((fem.FEM_OP_BP30, 3, 2, 2, 1, 800))
    items, refs = _build(specs, bases)
    batch = fem.Batch(items)
    batch.config = {"threads": 512, "group": 2, "order": 0, "layout": layout}
    batch.apply()
    torch.cuda.synchronize()
    for (op, b, geo, lam, q, out), (ref, v, _), spec in zip(items, refs, specs):
        if op == fem.FEM_OP_BP35 and b.N <= 9:
            pt = fem.fem_bp35_apply_layout(b, geo, lam, q, fem.FEM_LAYOUT_POINTS)
            assert torch.equal(out, pt), spec
            G, _ = oracle.geofacs(b.N, oracle.KIND_BP35, v)
            o = oracle.bp35(b.N, G, lam, q.cpu().numpy())
            assert np.abs(out.cpu().numpy() - o).max() / np.abs(o).max() < 1e-12, spec
        elif op == fem.FEM_OP_BP30 and layout & fem.FEM_BATCH_POINTS30:
            assert torch.equal(out, fem.fem_bp30_apply_layout(b, geo, lam, q, fem.FEM_LAYOUT_POINTS)), spec
        else:
            assert torch.equal(out, ref), spec


def test_full_size_batch_workload():
    """The benchmark's batch in full: 64 jittered meshes, N uniform in
    2..10, E log-uniform in 64..8192 (108,835 elements), BP3.5 and BP3.0 on
    each.  The tuned persistent launch and its graph replay equal the
    per-mesh calls in the tuned layouts bit for bit on every mesh, and
    sampled elements of every mesh match the oracle to 1e-12."""
    import torch
    fem = _fem()
    w = fem_synth.batch_workload()
    assert len(w) == 64 and sum(s["E"] for s in w) == 108835
    bases = {N: fem.fem_basis_setup(N) for N in sorted({s["N"] for s in w})}
    items, meta = [], []
    for s in w:
        b = bases[s["N"]]
        v = fem_synth.box_mesh(s["nx"], s["ny"], s["nz"], jitter=0.1, seed=s["mesh_seed"])
        q = _dev(fem_synth.field(s["mesh_seed"] + 7, s["E"], (s["N"] + 1) ** 3))
        for op, kind in ((fem.FEM_OP_BP35, fem.FEM_GEO_BP35), (fem.FEM_OP_BP30, fem.FEM_GEO_BP30)):
            g = fem.fem_mesh_geofacs(b, kind, _dev(v))
            items.append((op, b, g, 1.0, q, torch.full_like(q, float("nan"))))
            meta.append((s, v))
    batch = fem.Batch(items)
    batch.tune(reps=2)
    cfg = batch.config

    def per_mesh(op, b, g, q):
        pts = (op == fem.FEM_OP_BP35 and b.N <= 9 and cfg["layout"] & fem.FEM_BATCH_POINTS35) or \
              (op == fem.FEM_OP_BP30 and b.N <= 8 and cfg["layout"] & fem.FEM_BATCH_POINTS30)
        lay = fem.FEM_LAYOUT_POINTS if pts else fem.FEM_LAYOUT_LINES
        f = fem.fem_bp35_apply_layout if op == fem.FEM_OP_BP35 else fem.fem_bp30_apply_layout
        return f(b, g, 1.0, q, lay)

    rng = np.random.default_rng(5)
    for launch in (batch.apply, batch.graph_launch):
        for it in items:
            it[5].fill_(float("nan"))
        launch()
        torch.cuda.synchronize()
        for (op, b, g, lam, q, out), (s, v) in zip(items, meta):
            assert torch.equal(out, per_mesh(op, b, g, q)), (s, op, cfg)
    for (op, b, g, lam, q, out), (s, v) in zip(items, meta):
        pick = np.unique(np.concatenate([rng.choice(s["E"], 2, replace=False), [0, s["E"] - 1]]))
        kind = oracle.KIND_BP35 if op == fem.FEM_OP_BP35 else oracle.KIND_BP30
        G, _ = oracle.geofacs(b.N, kind, v[pick])
        ref = (oracle.bp35 if op == fem.FEM_OP_BP35 else oracle.bp30)(b.N, G, 1.0, q[pick].cpu().numpy())
        got = out[torch.from_numpy(pick).cuda()].cpu().numpy()
        assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12, (s, op)
    batch.free()


def test_batch_rejects_bad_items(bases):
    import torch
    fem = _fem()
    b11 = fem.fem_basis_setup(11)
    q = torch.zeros((1, 12 ** 3), dtype=torch.float64, device="cuda")
    g = torch.zeros((1, 7, 12 ** 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fem.FemError):
        fem.Batch([(fem.FEM_OP_BP35, b11, g, 1.0, q, torch.zeros_like(q))])
    with pytest.raises(fem.FemError):  # output aliasing the input
        b2 = bases[2]
        q2 = torch.zeros((1, 27), dtype=torch.float64, device="cuda")
        fem.Batch([(fem.FEM_OP_BP35, b2, torch.zeros((1, 7, 27), dtype=torch.float64, device="cuda"), 1.0, q2, q2)])
    empty = fem.Batch([])
    empty.apply()
    torch.cuda.synchronize()

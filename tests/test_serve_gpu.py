"""The continuous-batching solve server: each request's result is the same
bits alone and in the mix, the results meet their tolerance and agree with
the oracle's solve, and admission respects the HBM budget."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def _fem():
    import paper_1711_00903_gb300 as fem
    return fem


def _requests():
    out = []
    # last column: 0 FP64, 1 mixed (FP32 factors), 2 mixed with FP16 factors
    specs = [(2, 2, 2, 2, 0), (3, 3, 2, 2, 1), (3, 4, 2, 1, 0), (2, 5, 3, 2, 2), (3, 2, 1, 3, 1), (2, 6, 2, 2, 0),
             (3, 3, 2, 1, 2), (2, 7, 2, 2, 2)]
    for k, (op, N, nx, ny, mixed) in enumerate(specs):
        v = fem_synth.box_mesh(nx, ny, 2, jitter=0.1, seed=700 + k)
        rhs = fem_synth.field(800 + k, v.shape[0], (N + 1) ** 3)
        out.append((op, N, v, rhs, 0.5 + k % 2, mixed))
    return out


def _run(server, reqs, one_at_a_time, tol=1e-9):
    fem = _fem()
    ids = []
    for op, N, v, rhs, lam, mixed in reqs:
        mode = (fem.FEM_PCG_FP64, fem.FEM_PCG_MIXED, fem.FEM_PCG_MIXED16)[mixed]
        rid, x = server.submit(op, N, v, rhs, lam=lam, mode=mode, tol=tol)
        ids.append((rid, x))
        if one_at_a_time:
            server.drain()
    server.drain()
    return [(x, server.poll(rid)) for rid, x in ids]


def test_same_bits_alone_and_in_the_mix():
    fem = _fem()
    reqs = _requests()
    alone = _run(fem.Server(max_active=1), reqs, one_at_a_time=True)
    mixed = _run(fem.Server(max_active=8), reqs, one_at_a_time=False)
    for (xa, ra), (xm, rm), req in zip(alone, mixed, reqs):
        assert ra["state"] == rm["state"] == fem.FEM_REQ_DONE
        assert np.array_equal(xa, xm), req[:2]
        assert ra["iters"] == rm["iters"] and ra["relres"] == rm["relres"]
        assert rm["relres"] <= 1e-9


def test_results_against_the_oracle():
    fem = _fem()
    reqs = _requests()
    res = _run(fem.Server(max_active=4), reqs, one_at_a_time=False, tol=1e-11)
    for (x, r), (op, N, v, rhs, lam, mixed) in zip(res, reqs):
        if op == 2:
            G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
            xo, _, _ = oracle.pcg_bp35(N, G, lam, rhs, tol=1e-12)
            Ax = oracle.bp35(N, G, lam, x)
        else:
            G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
            xo, _, _ = oracle.pcg_bp30(N, G, lam, rhs, tol=1e-12)
            Ax = oracle.bp30(N, G, lam, x)
        assert np.linalg.norm(rhs - Ax) / np.linalg.norm(rhs) <= 2e-11
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-7


def test_admission_under_the_budget():
    fem = _fem()
    reqs = _requests()[:3]
    # a budget below any request's footprint: every request fails cleanly
    s = fem.Server(hbm_budget=1024, max_active=4)
    res = _run(s, reqs, one_at_a_time=False)
    for x, r in res:
        assert r["state"] == fem.FEM_REQ_FAILED and r["status"] == fem.FEM_ENOMEM
    # a budget that holds one request at a time: they run one after another
    big = max(r["bytes"] for _, r in res)
    s = fem.Server(hbm_budget=big + big // 2, max_active=4)
    res = _run(s, reqs, one_at_a_time=False)
    assert all(r["state"] == fem.FEM_REQ_DONE for _, r in res)
    for (_, a), (_, b) in zip(res, res[1:]):
        assert b["t_admit"] >= a["t_done"]
    assert s.in_use() == 0
    with pytest.raises(fem.FemError):
        s.poll(12345)


def _est_work(op, N, E, mixed, tol):
    """The server's work estimate for least-work-first admission (restated
    from its documented formula)."""
    w = E ** (4.0 / 3.0) * (N + 1) ** 3 * N * np.log(1.0 / tol)
    return w * (2.5 if op == 3 else 1.0) * (0.15 if mixed else 1.0)


def test_shortest_first_admission_order_and_same_bits():
    """With one slot and every request queued before the first progress
    call, FEM_SERVE_SHORTEST admits in increasing estimated work (ties by
    arrival), and each result is the same bits as under FIFO."""
    fem = _fem()
    reqs = _requests()
    fifo = _run(fem.Server(max_active=8), reqs, one_at_a_time=False)
    srv = fem.Server(max_active=1, policy=fem.FEM_SERVE_SHORTEST)
    sjf = _run(srv, reqs, one_at_a_time=False)
    for (xa, ra), (xs, rs) in zip(fifo, sjf):
        assert rs["state"] == fem.FEM_REQ_DONE
        assert np.array_equal(xa, xs)
    work = [_est_work(op, N, v.shape[0], mixed, 1e-9) for op, N, v, rhs, lam, mixed in reqs]
    order = sorted(range(len(reqs)), key=lambda k: (work[k], k))
    admitted = sorted(range(len(reqs)), key=lambda k: sjf[k][1]["t_admit"])
    assert admitted == order
    with pytest.raises(fem.FemError):
        fem.Server(policy=7)

"""Failure paths of the solver and the server, made on the host (no GPU
fault, no kernel left waiting): a device wait that gives up surfaces as
FEM_ETIMEDOUT through the public solve, a non-finite right-hand side as
FEM_EBREAKDOWN, and in the server a failed, cancelled or late request
leaves every other request's bits unchanged; the least-work-first policy
ages its queue so a large request is not starved."""
import time

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


def _system(op, N, nx=2):
    v = fem_synth.box_mesh(nx)
    kind = oracle.KIND_BP35 if op == 2 else oracle.KIND_BP30
    G, _ = oracle.geofacs(N, kind, v)
    b = fem_synth.field(11, v.shape[0], (N + 1) ** 3)
    return G, b


@pytest.mark.parametrize("op,mode", [(2, 0), (2, 1), (2, 2), (2, 3), (3, 1), (3, 3)],
                         ids=["bp35-fp64", "bp35-mixed", "bp35-mixed16", "bp35-mixed_tc", "bp30-mixed",
                              "bp30-mixed_tc"])
def test_wait_failure_surfaces_as_etimedout(op, mode):
    """The injected report (the status word a stream kernel writes when its
    bounded wait gives up) ends the solve with FEM_ETIMEDOUT; the next solve
    on the same context starts clean and gives the bits of a solve that
    never saw the fault."""
    import torch
    fem = _fem()
    N = 5  # FP32 and FP16-factor BP3.5 run the TMA stream kernel here
    G, b = _system(op, N)
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, mode, op=op)
    x_ref, _, code = s.solve(_dev(b), tol=1e-10)
    assert code == fem.FEM_OK
    s.inject_fault(fem.FEM_FAULT_WAIT_TIMEOUT)
    _, info, code = s.solve(_dev(b), tol=1e-10, raise_on_error=False)
    assert code == fem.FEM_ETIMEDOUT
    x2, _, code = s.solve(_dev(b), tol=1e-10)
    assert code == fem.FEM_OK and torch.equal(x2, x_ref)
    with pytest.raises(fem.FemError):
        s.inject_fault(7)  # unknown fault kind


def test_wait_selftest_reports_through_the_status_word():
    fem = _fem()
    gave_up, code = fem.fem_wait_selftest()
    assert gave_up == 2 and code == fem.FEM_ETIMEDOUT


@pytest.mark.parametrize("op,mode", [(2, 0), (2, 1), (2, 2), (3, 0), (3, 3)],
                         ids=["bp35-fp64", "bp35-mixed", "bp35-mixed16", "bp30-fp64", "bp30-mixed_tc"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_rhs_is_a_breakdown(op, mode, bad):
    fem = _fem()
    N = 4
    G, b = _system(op, N)
    b[1, 7] = bad
    basis = fem.fem_basis_setup(N)
    s = fem.fem_pcg_create(basis, _dev(G), 1.0, mode, op=op)
    _, _, code = s.solve(_dev(b), tol=1e-10, raise_on_error=False)
    assert code == fem.FEM_EBREAKDOWN
    b[1, 7] = 0.5  # the context stays usable
    _, _, code = s.solve(_dev(b), tol=1e-10)
    assert code == fem.FEM_OK


def _requests():
    out = []
    specs = [(2, 2, 2, 2, 0), (3, 3, 2, 2, 1), (3, 4, 2, 1, 0), (2, 5, 3, 2, 2), (3, 2, 1, 3, 3), (2, 6, 2, 2, 0),
             (3, 3, 2, 1, 2), (2, 7, 2, 2, 1)]
    for k, (op, N, nx, ny, mode) in enumerate(specs):
        v = fem_synth.box_mesh(nx, ny, 2, jitter=0.1, seed=900 + k)
        rhs = fem_synth.field(950 + k, v.shape[0], (N + 1) ** 3)
        out.append((op, N, v, rhs, mode))
    return out


def _submit(srv, reqs, tol=1e-9):
    return [srv.submit(op, N, v, rhs, lam=1.0, mode=mode, tol=tol) for op, N, v, rhs, mode in reqs]


def test_server_failed_request_leaves_the_others_bits():
    """A request with a NaN in its right-hand side fails (FEM_EBREAKDOWN)
    in the middle of the mix; every other request returns the bits it
    returns alone."""
    fem = _fem()
    reqs = _requests()
    alone = []
    srv = fem.Server(max_active=1)
    for r in reqs:
        rid, x = _submit(srv, [r])[0]
        srv.drain()
        assert srv.poll(rid)["state"] == fem.FEM_REQ_DONE
        alone.append(x)
    bad = list(reqs[3])
    bad[3] = bad[3].copy()
    bad[3][0, 0] = np.nan
    mix_reqs = reqs[:4] + [tuple(bad)] + reqs[4:]
    srv = fem.Server(max_active=8)
    ids = _submit(srv, mix_reqs)
    srv.drain()
    res = [srv.poll(rid) for rid, _ in ids]
    assert res[4]["state"] == fem.FEM_REQ_FAILED and res[4]["status"] == fem.FEM_EBREAKDOWN
    others = [(r, x) for k, (r, (_, x)) in enumerate(zip(res, ids)) if k != 4]
    for (r, x), xa in zip(others, alone):
        assert r["state"] == fem.FEM_REQ_DONE
        assert np.array_equal(x, xa)


def test_server_cancel_queued_and_running():
    fem = _fem()
    reqs = _requests()
    srv = fem.Server(max_active=2)
    ids = _submit(srv, reqs)
    srv.progress()  # two admitted, six queued
    running = [rid for rid, _ in ids if srv.poll(rid)["state"] == fem.FEM_REQ_RUNNING]
    queued = [rid for rid, _ in ids if srv.poll(rid)["state"] == fem.FEM_REQ_QUEUED]
    assert running and queued
    srv.cancel(queued[-1])
    r = srv.poll(queued[-1])
    assert r["state"] == fem.FEM_REQ_FAILED and r["status"] == fem.FEM_ECANCELED
    srv.cancel(running[0])
    srv.drain()
    r = srv.poll(running[0])
    assert r["state"] in (fem.FEM_REQ_FAILED, fem.FEM_REQ_DONE)  # DONE if it had already finished
    if r["state"] == fem.FEM_REQ_FAILED:
        assert r["status"] == fem.FEM_ECANCELED
    assert srv.in_use() == 0
    # every request not cancelled finished, with the bits of a solve alone
    alone = fem.Server(max_active=1)
    for (rid, x), req in zip(ids, reqs):
        if rid in (queued[-1], running[0]):
            continue
        assert srv.poll(rid)["state"] == fem.FEM_REQ_DONE
        rid2, x2 = _submit(alone, [req])[0]
        alone.drain()
        assert np.array_equal(x, x2)
    with pytest.raises(fem.FemError):
        srv.cancel(10 ** 9)


def test_server_wait_deadline():
    fem = _fem()
    srv = fem.Server(max_active=1)
    v = fem_synth.box_mesh(6)
    N = 6
    rhs = fem_synth.field(12, v.shape[0], (N + 1) ** 3)
    rid, x = srv.submit(3, N, v, rhs, lam=1.0, mode=fem.FEM_PCG_FP64, tol=1e-11)
    res, code = srv.wait(rid, 0.0)  # a deadline already passed
    assert code == fem.FEM_ETIMEDOUT and res["state"] in (fem.FEM_REQ_QUEUED, fem.FEM_REQ_RUNNING)
    res, code = srv.wait(rid, 600.0)
    assert code == fem.FEM_OK and res["state"] == fem.FEM_REQ_DONE and res["relres"] <= 1e-11


def _stream_behind_large(fem, max_wait_s, duration=1.5):
    """One small request running, a large one queued behind it, then small
    requests arriving for `duration` seconds; returns the large request's
    wait from submission to admission."""
    srv = fem.Server(max_active=1, policy=fem.FEM_SERVE_SHORTEST, max_wait_s=max_wait_s)
    small_v = fem_synth.box_mesh(1)
    small_rhs = fem_synth.field(13, 1, 27)
    srv.submit(2, 2, small_v, small_rhs, lam=1.0, mode=fem.FEM_PCG_FP64, tol=1e-8)
    srv.progress()
    big_v = fem_synth.box_mesh(6)
    big_rhs = fem_synth.field(14, big_v.shape[0], 8 ** 3)
    big, _ = srv.submit(2, 7, big_v, big_rhs, lam=1.0, mode=fem.FEM_PCG_FP64, tol=1e-9)
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < duration:
        srv.submit(2, 2, small_v, small_rhs, lam=1.0, mode=fem.FEM_PCG_FP64, tol=1e-8)
        for _ in range(4):
            srv.progress()
    srv.drain()
    r = srv.poll(big)
    assert r["state"] == fem.FEM_REQ_DONE
    wait = r["t_admit"] - r["t_submit"]
    srv.free()
    return wait


def test_least_work_first_ages_its_queue():
    """Without aging (a 100 s bound) the large request waits for the whole
    stream of small ones; with a 0.1 s bound it is admitted within the bound
    plus the small solve in flight."""
    fem = _fem()
    starved = _stream_behind_large(fem, 100.0)
    aged = _stream_behind_large(fem, 0.1)
    assert starved >= 1.0
    assert aged <= 0.6

"""Host logic of the multi-rank bench on CPU (gloo, world size 2): each rank
builds its own replica of the workload (same mesh recipe, its own field
stream), and the timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        verts, q = bench.workload_arrays(2, 3, r)
        bench.barrier(w)
        t = bench.reduce_max(float(10 + r), w)
        out[rank] = (t, float(verts.sum()), float(q[0, 0]), w)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0          # max over ranks
    assert res[0][1] == res[1][1]                  # same mesh recipe
    assert res[0][2] != res[1][2]                  # each rank its own field
    assert res[0][3] == res[1][3] == world


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    v, q = bench.workload_arrays(1, 2, 0)
    assert v.shape == (8, 8, 3) and q.shape == (8, 8)
    assert np.all(np.abs(q) <= 1.0)

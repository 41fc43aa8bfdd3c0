"""Failure detection of the device waits, without a fault: a kernel whose
mbarrier wait can never complete gives up after the wait's limit, counts
itself and returns, and the context stays usable for the TMA stream
kernels that rely on the same bounded wait."""
import numpy as np
import pytest

import fem_synth
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import torch
    import paper_1711_00903_gb300 as fem
    gave_up, code = fem.fem_wait_selftest()
    assert gave_up == 2  # both warps of the block gave up
    assert code == fem.FEM_ETIMEDOUT  # and the block reported it through its status word
    # the same process then runs the stream kernel normally
    fem.fem_wait_timeouts(reset=True)
    N = 7
    v = fem_synth.box_mesh(3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    q32 = fem_synth.field(5, v.shape[0], (N + 1) ** 3).astype(np.float32)
    ref = oracle.bp35(N, G.astype(np.float32).astype(np.float64), 1.0, q32.astype(np.float64))
    b = fem.fem_basis_setup(N)
    got = fem.fem_bp35_apply_f32(b, torch.from_numpy(G.astype(np.float32)).cuda(), 1.0,
                                 torch.from_numpy(q32).cuda()).cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-5
    assert fem.fem_wait_timeouts() == 0

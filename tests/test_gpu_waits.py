"""The bounded device-side wait of the FP32 tile gather, made to run out.

Each block of the gather stages its tile by asynchronous copies completed on
a shared-memory barrier, and one thread waits for it for a bounded time.
``erpp_debug_set_wait(stall=1)`` makes every such block, once its copies have
landed, also wait on a barrier that nothing completes: the wait runs out with
no copy in flight, the block records ERPP_ETIMEOUT and returns.  The test
checks that erpp_check reports it, that the context stays usable, and that
the next gather matches the oracle again.
"""

import dataclasses

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def erpp(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_6969_gb300 as pkg
    return pkg


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_gather_wait_runs_out_then_recovers(erpp, oracle_lib):
    import torch
    # rows of a multiple of 4 floats: every tile is staged by a TMA box or by
    # bulk row copies, both completed on the barrier the block waits for
    w = dataclasses.replace(I.CFG_SMALL, n=(72, 40, 20),
                            L=(2 * np.pi, 2 * np.pi * 40 / 72, 2 * np.pi * 20 / 72))
    p = w.params()
    grid, _ = I.make_grid(w)
    x_np = I.uniform_positions(2000, w.L, 5)
    x = torch.as_tensor(x_np).cuda().contiguous()
    u = torch.as_tensor(grid, dtype=torch.float32).cuda().contiguous()
    ctx = erpp.Context(p, precision="fp32")
    assert ctx.tiling()[0] == 4
    with pytest.raises(erpp.ErppError):
        ctx.debug_set_wait(limit_ns=10, stall=False)  # below the smallest limit
    ctx.debug_set_wait(limit_ns=2_000_000, stall=True)
    ctx.interpolate(u, x)
    with pytest.raises(erpp.ErppError) as ei:
        ctx.check()
    assert ei.value.status == 6  # ERPP_ETIMEOUT
    ctx.check()  # reported once, then cleared
    ctx.debug_set_wait(0, False)
    ref = oracle_lib.gather(p, x_np, grid)
    for _ in range(2):
        up = ctx.interpolate(u, x)
        ctx.check()
        assert _rel(up.cpu().numpy(), ref) < 1e-5
    torch.cuda.synchronize()
    ctx.close()

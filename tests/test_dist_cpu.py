"""The multi-rank host path of the benchmark (independent boxes per rank,
max-over-ranks timing) with two gloo ranks on the CPU."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1405_6969_gb300 import dist as D
    ws, r, local = D.env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    D.barrier()
    t = D.max_over_ranks(1.0 + 0.5 * r)  # rank 1 is slower
    out[r] = (D.box_seed(0, r), D.batched_seed0(r), t, D.aggregate_rate(100.0, ws, t))
    D.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world                       # independent boxes
    assert out[0][1] == 0 and out[1][1] == 64        # disjoint batches of 64 seeds
    assert out[0][2] == out[1][2] == pytest.approx(1.5)   # slowest rank's time
    assert out[0][3] == pytest.approx(2 * 100.0 / 1.5)    # whole-job rate


def test_single_process_defaults(monkeypatch):
    from paper_1405_6969_gb300 import dist as D
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert D.env() == (1, 0, 0)
    assert D.max_over_ranks(3.0) == 3.0

"""The slab domain decomposition with the CUDA library as each rank's local
arithmetic (slab.ContextCompute), on one GPU: two or three ranks run as host
threads that exchange planes, ghost particles and migrants through queues (no
kernel waits on another rank; every exchange happens on the host between
launches).  The union of the slabs' sources and the particles after three
coupled steps match the single-box FP64 oracle step: 1e-12 (FP64 contexts)
and 1e-5 relative L2 (FP32 contexts)."""

import math
import queue
import threading

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


class ThreadComm:
    """Neighbour exchanges between ranks that are threads of one process."""

    def __init__(self, geom, boxes, barrier, sums):
        self.geom, self.boxes, self.barrier, self.sums = geom, boxes, barrier, sums

    def exchange(self, to_lower, to_upper):
        g = self.geom
        self.boxes[(g.rank, g.lower, "down")].put(to_lower)
        self.boxes[(g.rank, g.upper, "up")].put(to_upper)
        from_lower = self.boxes[(g.lower, g.rank, "up")].get(timeout=120)
        from_upper = self.boxes[(g.upper, g.rank, "down")].get(timeout=120)
        return from_lower, from_upper

    def allreduce_sum(self, t):
        self.sums[self.geom.rank] = t.clone()
        self.barrier.wait(timeout=120)
        total = sum(self.sums[r].to(t.device) for r in range(self.geom.world))
        self.barrier.wait(timeout=120)
        return total


def _workload():
    w = I.CFG_SMALL.scaled("slab", (24, 16, 48), 800,
                           L=(2 * math.pi * 24 / 48, 2 * math.pi * 16 / 48, 2 * math.pi))
    w = I.dataclasses.replace(w, dt=0.04, shear_rate=0.5)
    return w, w.params(gravity=(0.0, 0.0, -2.0))


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("world", [2, 3])
def test_gpu_slabs_match_single_box(erpp, oracle_lib, world, precision):
    import torch
    from paper_1405_6969_gb300 import slab as SL
    steps = 3
    w, p = _workload()
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    dt = torch.float32 if precision == "fp32" else torch.float64
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    full = SL.SlabState(t(st.x), t(st.v), t(st.x_prev), t(st.D), t(st.radius), t(st.rho_p),
                        torch.arange(st.n, dtype=torch.float64, device="cuda"))
    u = torch.as_tensor(grid, dtype=dt).cuda()
    boxes = {(a, b, d): queue.Queue() for a in range(world) for b in range(world)
             for d in ("up", "down")}
    barrier = threading.Barrier(world)
    sums = {}
    out, errors = {}, []

    def rank_main(rank):
        try:
            torch.cuda.set_device(0)
            geom = SL.SlabGeometry(p, world, rank)
            comm = ThreadComm(geom, boxes, barrier, sums)
            comp = SL.ContextCompute(geom, precision=precision)
            mine = SL.split_particles(geom, full)
            u_own = SL.own_planes(geom, u)
            for k in range(steps):
                S_own, mine = SL.slab_step(geom, comm, comp, u_own, mine, first_step=(k == 0))
            comp.ctx.check()
            mom = SL.slab_momentum(geom, comm, S_own, mine, p)
            torch.cuda.synchronize()
            out[rank] = (geom.z0, S_own.double().cpu().numpy(), mine.records().cpu().numpy(),
                         mom.cpu().numpy())
            comp.close()
        except Exception as e:  # reported by the main thread
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(300)
    assert not errors, errors
    ref = st.copy()
    for k in range(steps):
        S_ref = oracle_lib.step(p, grid, ref, first_step=(k == 0))
    parts = sorted((out[r] for r in range(world)), key=lambda o: o[0])
    S = np.concatenate([o[1] for o in parts], axis=1)
    rec = np.concatenate([o[2] for o in parts], axis=1)
    ids = rec[14].astype(int)
    assert sorted(ids.tolist()) == list(range(ref.n))
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert _rel(S, S_ref) < tol
    for name, rows in (("v", slice(3, 6)), ("D", slice(9, 12))):
        got = np.empty((3, ref.n))
        got[:, ids] = rec[rows]
        assert _rel(got, getattr(ref, name)) < tol, name
    Pg, Pp = oracle_lib.momentum(p, ref.x_prev, ref.D, S_ref)
    # the all-reduced impulse of the slabs against the single box's (FP32: the
    # forces carry the FP32 path's rounding)
    mtol = 1e-10 if precision == "fp64" else tol
    np.testing.assert_allclose(parts[0][3][3:], Pp, rtol=mtol)
    np.testing.assert_allclose(parts[0][3][:3], Pg, rtol=tol, atol=tol * np.abs(Pp).max())

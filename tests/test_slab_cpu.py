"""The slab domain decomposition (paper_1405_6969_gb300.slab) on gloo ranks on
the CPU: one periodic box cut into two or three z-slabs, each rank stepping
its slab with the FP64 oracle as the local arithmetic (ghost planes of the
fluid field, neighbours' particles near the faces, migration, the momentum
all-reduce).  The union of the slabs' sources and the particles' updated
state after three coupled steps equal the single-box oracle's, to rounding;
some particles change slab on the way."""

import math
import os
import socket

import numpy as np
import pytest

import erpp_inputs as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    # isotropic spacing, 48 planes in z so that two or three slabs each keep
    # more planes than the ghost depth; a large dt so that particles migrate
    w = I.CFG_SMALL.scaled("slab", (20, 16, 48), 700,
                           L=(2 * math.pi * 20 / 48, 2 * math.pi * 16 / 48, 2 * math.pi))
    w = I.dataclasses.replace(w, dt=0.04, shear_rate=0.5)
    return w, w.params(gravity=(0.0, 0.0, -2.0))


class _OracleCompute:
    """The oracle on a rank's local box (test stand-in for the GPU context)."""

    def __init__(self, p):
        import oracle
        self.o, self.p = oracle, p

    def gather(self, u_loc, x):
        import torch
        return torch.from_numpy(self.o.gather(self.p, x.numpy(), u_loc.numpy()))

    def advance(self, up, ls, first_step):
        class S:  # numpy views of the state's tensors, updated in place
            pass
        s = S()
        for k in ("x", "v", "x_prev", "D", "radius", "rho_p"):
            setattr(s, k, getattr(ls, k).numpy())
        s.n = ls.x.shape[1]
        self.o.advance(self.p, up.numpy(), s, first_step=first_step)

    def scatter(self, x, D):
        import torch
        return torch.from_numpy(self.o.scatter(self.p, x.numpy(), D.numpy()))


def _worker(rank, world, port, steps, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1405_6969_gb300 import slab as SL
        w, p = _workload()
        grid, field = I.make_grid(w)
        st = I.make_particles(w, field)
        geom = SL.SlabGeometry(p, world, rank)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a))  # noqa: E731
        full = SL.SlabState(t(st.x), t(st.v), t(st.x_prev), t(st.D), t(st.radius), t(st.rho_p),
                            torch.arange(st.n, dtype=torch.float64))
        mine = SL.split_particles(geom, full)
        first_ids = set(mine.ids.numpy().astype(int).tolist())
        u_own = SL.own_planes(geom, t(grid))
        comm = SL.TorchComm(geom)
        comp = _OracleCompute(geom.local_params)
        for k in range(steps):
            S_own, mine = SL.slab_step(geom, comm, comp, u_own, mine, first_step=(k == 0))
        mom = SL.slab_momentum(geom, comm, S_own, mine, p)
        moved = len(first_ids ^ set(mine.ids.numpy().astype(int).tolist()))
        out[rank] = (geom.z0, S_own.numpy(), mine.records().numpy(), mom.numpy(), moved)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_single_box(oracle_lib, world):
    import torch.multiprocessing as mp
    steps = 3
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    # the single box, stepped by the oracle
    w, p = _workload()
    grid, field = I.make_grid(w)
    ref = I.make_particles(w, field)
    for k in range(steps):
        S_ref = oracle_lib.step(p, grid, ref, first_step=(k == 0))
    parts = sorted((out[r] for r in range(world)), key=lambda o: o[0])
    S = np.concatenate([o[1] for o in parts], axis=1)
    scale = np.abs(S_ref).max()
    np.testing.assert_allclose(S, S_ref, rtol=0, atol=1e-12 * scale)
    rec = np.concatenate([o[2] for o in parts], axis=1)
    ids = rec[14].astype(int)
    assert sorted(ids.tolist()) == list(range(ref.n))  # every particle once
    for name, rows in (("x", slice(0, 3)), ("v", slice(3, 6)), ("x_prev", slice(6, 9)),
                       ("D", slice(9, 12))):
        got = np.empty((3, ref.n))
        got[:, ids] = rec[rows]
        want = getattr(ref, name)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * max(np.abs(want).max(), 1e-300),
                                   err_msg=name)
    # momentum: one all-reduce, the same on every rank, equal to the oracle's
    Pg, Pp = oracle_lib.momentum(p, ref.x_prev, ref.D, S_ref)
    for o in parts:
        np.testing.assert_allclose(o[3][:3], Pg, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(o[3][3:], Pp, rtol=1e-10, atol=1e-14)
    assert sum(o[4] for o in parts) > 0  # particles changed slab


def test_slab_geometry_host():
    from paper_1405_6969_gb300 import slab as SL
    import torch
    _, p = _workload()
    g2 = [SL.SlabGeometry(p, 2, r) for r in range(2)]
    assert g2[0].bounds == [0, 24, 48] and g2[0].reach == 4 and g2[0].g == 9
    assert g2[0].lower == g2[0].upper == 1
    z = torch.tensor([0.0, 2 * math.pi * 23.99 / 48, 2 * math.pi * 24 / 48, 2 * math.pi - 1e-9],
                     dtype=torch.float64)
    assert g2[0].owner(z).tolist() == [0, 0, 1, 1]
    np.testing.assert_allclose(g2[1].to_global(g2[1].to_local(z)), z, atol=1e-12)
    with pytest.raises(ValueError):
        SL.SlabGeometry(p, 6, 0)  # slabs of 8 planes, thinner than the ghost depth

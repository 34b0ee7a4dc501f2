"""Slab domain decomposition of one periodic box over several ranks.

The box is cut along z into contiguous slabs of node planes, one per rank.
Each rank holds its planes of the fluid field and the particles whose home
cell (floor(z N_z / L_z)) lies in them, and computes, per coupling step:

1. the fluid field on a local periodic box made of its planes and ``g``
   ghost planes on each side, filled from the neighbouring slabs (one plane
   exchange);
2. the gather, self-disturbance removal, drag and advance of its own
   particles on that local box (the stencil of an own particle reaches at
   most ``reach`` planes beyond the slab);
3. the source of its own planes: the regularised source (Eq.
   ns_regularized_filtered) of its own particles and of the neighbours'
   particles whose stencils reach its planes (their positions x^n and forces
   D^n are exchanged first), computed on the local box and cut to the own
   planes -- every node is computed once, by its owner, from every particle
   that reaches it, so no halo of the source is added;
4. the migration of particles whose new position left the slab;
5. the momentum check (Sec. 3.1) as one all-reduce of six doubles.

The ghost depth ``g`` is at least twice the reach plus one, so that the
stencil of a neighbour's particle, which may extend ``reach`` planes beyond
the neighbour's own face, never wraps around the local box into the own
planes.  The paper gives no parallel layout of its own (Sec. 1 only calls the
method suited to massively parallel machines); this one is owner-computes
with one exchange per phase.

The local arithmetic is pluggable: ``ContextCompute`` runs the CUDA library
on the rank's GPU; a test may substitute any object with the same three
methods.  Exchanges go through ``TorchComm`` (torch.distributed point-to-point
sends: NCCL between GPUs, gloo between CPU processes) or any object with the
same ``exchange`` method.  Host logic only.
"""

from __future__ import annotations

import math

import torch

class SlabGeometry:
    """The z-slab of rank ``rank`` out of ``world`` for a parameter dict."""

    def __init__(self, params, world, rank):
        self.params = dict(params)
        self.world, self.rank = int(world), int(rank)
        n = [int(v) for v in params["n"]]
        L = [float(v) for v in params["L"]]
        self.nz, self.Lz = n[2], L[2]
        self.dz = self.Lz / self.nz
        sig = math.sqrt(2.0 * float(params["nu"]) * float(params["eps_R"]))
        cz = float(params["cutoff"]) * sig / self.dz
        self.reach = int(math.floor(cz)) + 1        # planes beyond the home cell
        self.g = 2 * self.reach + 1                 # ghost planes on each side
        self.bounds = [self.nz * r // self.world for r in range(self.world + 1)]
        self.z0, self.z1 = self.bounds[self.rank], self.bounds[self.rank + 1]
        if min(b - a for a, b in zip(self.bounds, self.bounds[1:])) < self.g:
            raise ValueError("every slab needs at least as many planes as the ghost depth "
                             f"({self.g}); use fewer ranks")
        self.ns = self.z1 - self.z0
        self.nz_loc = self.ns + 2 * self.g
        if self.nz_loc > self.nz:
            raise ValueError("the local box would exceed the box: use fewer ranks")
        self.lower = (self.rank - 1) % self.world
        self.upper = (self.rank + 1) % self.world
        # local plane 0 is global plane z0 - g
        self.shift = (self.z0 - self.g) * self.dz
        self.local_params = dict(self.params, n=(n[0], n[1], self.nz_loc),
                                 L=(L[0], L[1], self.nz_loc * self.dz))

    def cell(self, z):
        """Global home-cell plane of positions z (the kernels' s = z N / L)."""
        return torch.floor(z * (self.nz / self.Lz)).to(torch.int64) % self.nz

    def owner(self, z):
        """Rank owning each position."""
        c = self.cell(z)
        b = torch.as_tensor(self.bounds[1:-1], dtype=torch.int64, device=z.device)
        return torch.bucketize(c, b, right=True)

    def to_local(self, z):
        return torch.remainder(z - self.shift, self.Lz)

    def to_global(self, z):
        return torch.remainder(z + self.shift, self.Lz)


class TorchComm:
    """Exchanges with the two neighbouring slabs through torch.distributed
    point-to-point operations (every rank calls exchange in the same order)."""

    def __init__(self, geom):
        self.geom = geom

    def exchange(self, to_lower, to_upper):
        """Send two tensors (rows x columns, the column count may be 0) down
        and up; return what the lower and upper neighbours sent.  With two
        ranks both neighbours are the same rank."""
        import torch.distributed as dist
        g = self.geom
        dev = to_lower.device
        sizes = [torch.tensor([to_lower.shape[-1]], dtype=torch.int64, device=dev),
                 torch.tensor([to_upper.shape[-1]], dtype=torch.int64, device=dev)]
        got = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(2)]
        # the count sent down arrives as the upper neighbour's "from lower"
        ops = [dist.P2POp(dist.isend, sizes[0], g.lower, tag=1),
               dist.P2POp(dist.isend, sizes[1], g.upper, tag=2),
               dist.P2POp(dist.irecv, got[1], g.upper, tag=1),
               dist.P2POp(dist.irecv, got[0], g.lower, tag=2)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        shape = to_lower.shape[:-1]
        recv = [torch.empty(*shape, int(got[k].item()), dtype=to_lower.dtype, device=dev)
                for k in range(2)]
        ops = []
        if to_lower.shape[-1]:
            ops.append(dist.P2POp(dist.isend, to_lower.contiguous(), g.lower, tag=3))
        if to_upper.shape[-1]:
            ops.append(dist.P2POp(dist.isend, to_upper.contiguous(), g.upper, tag=4))
        if recv[1].shape[-1]:
            ops.append(dist.P2POp(dist.irecv, recv[1], g.upper, tag=3))
        if recv[0].shape[-1]:
            ops.append(dist.P2POp(dist.irecv, recv[0], g.lower, tag=4))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        return recv[0], recv[1]

    def allreduce_sum(self, t):
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t


class ContextCompute:
    """The local arithmetic of a rank on its GPU, through the CUDA library:
    an FP32 or FP64 context on the local box."""

    def __init__(self, geom, precision="fp32", **opts):
        from .erpp import Context
        self.ctx = Context(geom.local_params, precision=precision, **opts)
        self.grid_dtype = self.ctx.grid_dtype

    def gather(self, u_loc, x):
        return self.ctx.interpolate(u_loc, x)

    def advance(self, up, state, first_step):
        self.ctx.particle_advance(up, state, first_step=first_step)

    def scatter(self, x, D):
        return self.ctx.scatter_source(x, D)

    def close(self):
        self.ctx.close()


class SlabState:
    """A rank's own particles (global coordinates) and their global ids; the
    fields are [3, m] (x, v, x_prev, D) and [m] (radius, rho_p, id) tensors.
    A migrating record stacks them as 15 rows: x, v, x_prev, D, radius, rho_p,
    id."""

    def __init__(self, x, v, x_prev, D, radius, rho_p, ids):
        self.x, self.v, self.x_prev, self.D = x, v, x_prev, D
        self.radius, self.rho_p, self.ids = radius, rho_p, ids

    @property
    def n(self):
        return self.x.shape[1]

    def records(self, mask=None):
        rows = torch.cat([self.x, self.v, self.x_prev, self.D, self.radius[None],
                          self.rho_p[None], self.ids[None]], dim=0)
        return rows if mask is None else rows[:, mask]

    @staticmethod
    def from_records(r):
        return SlabState(r[0:3].contiguous(), r[3:6].contiguous(), r[6:9].contiguous(),
                         r[9:12].contiguous(), r[12].contiguous(), r[13].contiguous(),
                         r[14].contiguous())


def split_particles(geom, state):
    """This rank's share of a whole-box SlabState."""
    return SlabState.from_records(state.records(geom.owner(state.x[2]) == geom.rank))


def own_planes(geom, u):
    """This rank's planes of a whole-box grid field [3, nz, ny, nx]."""
    return u[:, geom.z0:geom.z1].contiguous()


def _local_state(geom, st):
    """The rank's particles as the library's ParticleState in local
    coordinates (z shifted so that local plane 0 is global plane z0 - g)."""
    from .erpp import ParticleState
    x = st.x.clone()
    xp = st.x_prev.clone()
    x[2] = geom.to_local(x[2])
    xp[2] = geom.to_local(xp[2])
    return ParticleState(x.contiguous(), st.v.clone(), xp.contiguous(), st.D.clone(),
                         st.radius.contiguous(), st.rho_p.contiguous())


def slab_step(geom, comm, compute, u_own, st, first_step=False):
    """One coupling step of this rank's slab.  u_own: its planes of the fluid
    field [3, ns, ny, nx] (held fixed); st: its SlabState (global
    coordinates, updated and migrated).  Returns (S_own [3, ns, ny, nx], the
    new SlabState)."""
    g = geom.g
    # 1. the fluid field on the local box: the bottom planes go down (the
    # lower neighbour's upper ghost), the top planes go up
    lo_planes, hi_planes = comm.exchange(u_own[:, :g].reshape(1, -1), u_own[:, -g:].reshape(1, -1))
    shape = (3, g) + tuple(u_own.shape[2:])
    u_loc = torch.cat([lo_planes.reshape(shape), u_own, hi_planes.reshape(shape)],
                      dim=1).contiguous()
    # 2. gather, removal, drag, advance of the own particles (local z)
    ls = _local_state(geom, st)
    if st.n:
        up = compute.gather(u_loc, ls.x)
        compute.advance(up, ls, first_step)
    # back to global coordinates (the advance may have wrapped in the local
    # box only through the ghost planes)
    x = ls.x.clone()
    xp = ls.x_prev.clone()
    x[2] = geom.to_global(x[2])
    xp[2] = geom.to_global(xp[2])
    st = SlabState(x, ls.v, xp, ls.D, st.radius, st.rho_p, st.ids)
    # 3. the neighbours' particles whose stencils reach this slab: positions
    # x^n (now x_prev) and forces D^n of particles within `reach` planes of a
    # face (with two ranks, both faces go to the same rank, once)
    c = geom.cell(st.x_prev[2])
    near_lo = ((c - geom.z0) % geom.nz) < geom.reach
    near_hi = ((geom.z1 - 1 - c) % geom.nz) < geom.reach
    rec = torch.cat([st.x_prev, st.D], dim=0)
    if geom.lower == geom.upper:
        to_lo, to_hi = rec[:, near_lo | near_hi], rec[:, :0]
    else:
        to_lo, to_hi = rec[:, near_lo], rec[:, near_hi]
    from_lo, from_hi = comm.exchange(to_lo, to_hi)
    xs = torch.cat([st.x_prev, from_lo[0:3], from_hi[0:3]], dim=1)
    Ds = torch.cat([st.D, from_lo[3:6], from_hi[3:6]], dim=1)
    xs = xs.clone()
    xs[2] = geom.to_local(xs[2])
    S_loc = compute.scatter(xs.contiguous(), Ds.contiguous())
    S_own = S_loc[:, g:g + geom.ns].contiguous()
    # 4. migration: particles whose new home cell left the slab
    own = geom.owner(st.x[2])
    keep = own == geom.rank
    recs = st.records()
    if geom.lower == geom.upper:
        out_lo, out_hi = recs[:, ~keep], recs[:, :0]
    else:
        out_lo, out_hi = recs[:, own == geom.lower], recs[:, own == geom.upper]
        if bool(((~keep) & (own != geom.lower) & (own != geom.upper)).any()):
            raise RuntimeError("a particle moved further than one slab in one step")
    in_lo, in_hi = comm.exchange(out_lo, out_hi)
    st = SlabState.from_records(torch.cat([recs[:, keep], in_lo, in_hi], dim=1))
    return S_own, st


def slab_momentum(geom, comm, S_own, st, params):
    """The impulse check of Sec. 3.1 over all ranks: (dV sum S, -(1/rho_f)
    sum D) in FP64, normalised weights (unit discrete mass), one all-reduce."""
    n = [int(v) for v in params["n"]]
    L = [float(v) for v in params["L"]]
    dV = (L[0] / n[0]) * (L[1] / n[1]) * (L[2] / n[2])
    out = torch.zeros(6, dtype=torch.float64, device=S_own.device)
    out[:3] = dV * S_own.double().sum(dim=(1, 2, 3))
    out[3:] = -(1.0 / float(params.get("rho_f", 1.0))) * st.D.sum(dim=1)
    return comm.allreduce_sum(out)

"""GPU parity at the benchmark's own sizes.

The homogeneous-shear-like box (4pi x 2pi x 2pi, 512 x 256 x 256 nodes,
1,000,000 particles, Stokes mix {0.1, 1, 10}, mass loading 0.4, mean shear
1) and the 256^3 box with 1M particles, in the launch configurations the
benchmark times (the default tiles, the autotuner's usual pick 16x2x256 and a
512-thread shape; the fixed-point and the compensated scatter; the three
ways of handling tile halos).  One coupling
step (gather, self removal, drag, Euler advance, scatter) against the FP64
oracle over every particle and every node:

* stencil windows bit-exact for all particles;
* the source S, the forces D and the velocities v within the FP32
  tolerance (1e-5 relative L2), x_prev bit-exact, x within the bound of the
  FP64 integration of those velocities;
* the step repeated from the same state bit-identical (fixed-point scatter).

The oracle runs on the host cores (``oracle.step_threads``: the unchanged
oracle step on particle chunks, partial sources summed), once per workload.
"""

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _threads():
    import os
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return max(1, min(8, n or 1))


_CACHE = {}


def _workload(name, oracle_lib):
    """Inputs and the oracle's step of one workload (computed once)."""
    if name not in _CACHE:
        _CACHE.clear()  # one full-size workload held at a time
        w = {"shear512": I.CFG_SHEAR, "cube256": I.CFG_CUBE256}[name]
        p = w.params(gravity=(0.0, -9.81, 0.0))
        grid, _ = I.make_grid(w)
        st = I.make_particles(w, None)
        ref = st.copy()
        S_ref = oracle_lib.step_threads(p, grid, ref, _threads(), first_step=False)
        _CACHE[name] = (w, p, grid, st, ref, S_ref)
    return _CACHE[name]


# (workload, tiling T_y x T_z x threads (0 = default), compensated scatter,
# scatter mode)
CASES = [
    ("shear512", (0, 0, 0), False, "merge"),
    ("shear512", (16, 2, 256), False, "merge"),
    ("shear512", (32, 2, 512), False, "merge"),
    ("shear512", (16, 2, 256), True, "merge"),
    ("shear512", (16, 2, 256), False, "xclip"),
    ("shear512", (16, 2, 256), True, "xclip"),
    ("shear512", (32, 2, 512), False, "cluster"),
    ("cube256", (0, 0, 0), False, "merge"),
    ("cube256", (16, 2, 256), False, "merge"),
    ("cube256", (16, 2, 256), True, "merge"),
    ("cube256", (16, 2, 256), False, "xclip"),
]


@pytest.mark.parametrize("name,tile,kahan,mode", CASES,
                         ids=[f"{c[0]}-{'x'.join(map(str, c[1]))}-"
                              f"{'kahan' if c[2] else 'fixed'}-{c[3]}" for c in CASES])
def test_full_size_step(erpp, oracle_lib, name, tile, kahan, mode):
    import torch
    w, p, grid, st, ref, S_ref = _workload(name, oracle_lib)
    ctx = erpp.Context(p, precision="fp32", kahan=kahan)
    ctx.set_scatter_mode(mode)
    if any(tile):
        ctx.set_tiling(*tile)
    assert ctx.tiling()[0] == 4
    x = torch.as_tensor(st.x).cuda().contiguous()
    if tile == (0, 0, 0) and not kahan:
        lo, hi = ctx.debug_windows(x)
        rlo, rhi = oracle_lib.windows(p, st.x)
        np.testing.assert_array_equal(lo.cpu().numpy(), rlo)
        np.testing.assert_array_equal(hi.cpu().numpy(), rhi)
        del lo, hi
    u = torch.as_tensor(grid, dtype=torch.float32).cuda().contiguous()
    ps = erpp.ParticleState.from_numpy(st)
    S = ctx.step(u, ps, first_step=False)
    ctx.check()
    errs = {"S": _rel(S.cpu().numpy(), S_ref), "D": _rel(ps.D.cpu().numpy(), ref.D),
            "v": _rel(ps.v.cpu().numpy(), ref.v)}
    print(f"\n{name} tiles {ctx.tiling()} kahan={kahan} {mode}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["S"] < TOL and errs["D"] < TOL and errs["v"] < TOL
    np.testing.assert_array_equal(ps.x_prev.cpu().numpy(), st.x)
    # x^(n+1) = x^n + dt v^n from the FP64 input velocity: FP64 rounding only
    dxp = np.abs(ps.x.cpu().numpy() - ref.x)
    dxp = np.minimum(dxp, np.array(w.L)[:, None] - dxp)
    assert dxp.max() < 1e-12 * 10 * max(w.L)
    if not kahan:
        # the same step again from the same state: the per-piece gather sums
        # added in piece order, the fixed-point scatter sums and the fixed
        # merge order give the same bits
        S1, D1 = S.clone(), ps.D.clone()
        ps = erpp.ParticleState.from_numpy(st)
        ctx.step(u, ps, S=S, first_step=False)
        ctx.check()
        assert torch.equal(S, S1) and torch.equal(ps.D, D1)
        del S1, D1
    del S, u, ps
    ctx.close()
    torch.cuda.empty_cache()

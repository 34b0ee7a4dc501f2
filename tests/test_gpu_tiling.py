"""GPU parity of every x/y-halo tile shape the autotuner may choose, and the
autotuner itself.  Tolerances as in the other parity tests (relative L2,
1e-5 FP32); expected values from the oracle."""

import dataclasses
import math

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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


CASES = [
    ("ragged_72x40x20", dataclasses.replace(I.CFG_SMALL, n=(72, 40, 20), kmax=3.0,
                                            L=(2 * math.pi, 2 * math.pi * 40 / 72,
                                               2 * math.pi * 20 / 72)), 3000),
    ("sigma1.5_48x44x30", dataclasses.replace(I.CFG_CLUSTERED, n=(48, 44, 30),
                                              L=(2 * math.pi, 2 * math.pi * 44 / 48,
                                                 2 * math.pi * 30 / 48),
                                              cluster_std=0.4), 2500),
]
TILES = [(16, 4, 256), (8, 4, 256), (16, 2, 256), (32, 2, 256), (8, 2, 256), (32, 1, 256),
         (5, 1, 256), (32, 4, 256), (16, 4, 512), (32, 2, 512), (8, 2, 512), (32, 1, 512)]


@pytest.mark.parametrize("tile", TILES, ids=["x".join(map(str, t)) for t in TILES])
@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_step_every_tiling(erpp, oracle_lib, name, w, npart, tile):
    import torch
    p = w.params(gravity=(0.0, -1.0, 0.0))
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field, n_particles=npart)
    ctx = erpp.Context(p, precision="fp32")
    ctx.set_tiling(*tile)
    design, W, ty, tz, nt = ctx.tiling()
    assert design == 4 and nt == tile[2]
    ps = erpp.ParticleState.from_numpy(st)
    S = ctx.step(cuda(grid, torch.float32), ps, first_step=False)
    ctx.check()
    ref = st.copy()
    S_ref = oracle_lib.step(p, grid, ref, first_step=False)
    assert rel(S.cpu().numpy(), S_ref) < 1e-5
    assert rel(ps.D.cpu().numpy(), ref.D) < 1e-5
    assert rel(ps.v.cpu().numpy(), ref.v) < 1e-5


def test_set_tiling_rejects_and_keeps_working(erpp, oracle_lib):
    w = I.CFG_SMALL
    ctx = erpp.Context(w.params(), precision="fp32")
    before = ctx.tiling()
    for bad in ((33, 4, 0), (16, 3, 0), (-1, 4, 0), (16, 4, 384)):
        with pytest.raises(erpp.ErppError):
            ctx.set_tiling(*bad)
    assert ctx.tiling() == before
    x = I.uniform_positions(500, w.L, 4)
    D = np.random.default_rng(5).standard_normal((3, 500))
    S = ctx.scatter_source(cuda(x), cuda(D))
    assert rel(S.cpu().numpy(), oracle_lib.scatter(w.params(), x, D)) < 1e-5


def test_autotune_picks_and_caches(erpp, oracle_lib, tmp_path):
    import torch
    from paper_1405_6969_gb300 import autotune
    w = dataclasses.replace(I.CFG_SMALL, n=(64, 48, 40), kmax=3.0,
                            L=(2 * math.pi, 2 * math.pi * 48 / 64, 2 * math.pi * 40 / 64))
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field, n_particles=5000)
    ctx = erpp.Context(w.params(), precision="fp32")
    u = cuda(grid, torch.float32)
    ps = erpp.ParticleState.from_numpy(st)
    x0 = ps.x.clone()
    path = str(tmp_path / "tune.json")
    r1 = autotune.tune(ctx, u, ps, steps=2, warmup=1, cache_path=path)
    # every shape with the merge scatter, the three fastest again with
    # clusters and with cut x-windows
    assert not r1["cached"] and len(r1["ms"]) == len(autotune.CANDIDATES) + 6
    assert r1["mode"] in ("merge", "cluster", "xclip") and ctx.scatter_mode() == r1["mode"]
    assert torch.equal(ps.x, x0)  # tuning works on copies of the state
    r2 = autotune.tune(ctx, u, ps, cache_path=path)
    assert r2["cached"] and r2["tile"] == r1["tile"] and r2["mode"] == r1["mode"]
    S = ctx.step(u, ps, first_step=False)
    ref = st.copy()
    S_ref = oracle_lib.step(w.params(), grid, ref, first_step=False)
    assert rel(S.cpu().numpy(), S_ref) < 1e-5

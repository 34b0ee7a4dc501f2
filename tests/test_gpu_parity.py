"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 over the whole output): 1e-5 for the FP32 kernels,
1e-12 for the FP64 kernels; stencil windows bit-exact.  Every input comes
from the seeded generators in ``erpp_inputs``; every expected value from
``oracle``.
"""

import dataclasses
import math

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


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


def grid_t(g, precision):
    import torch
    return cuda(g, torch.float32 if precision == "fp32" else torch.float64)


def rep(w, **kw):
    return dataclasses.replace(w, **kw)


# Grids chosen to span several tiles (32 x 16 x 8) with ragged last tiles,
# and small grids where one tile covers a whole periodic axis.
CASES = [
    ("cube32_uniform", rep(I.CFG_SMALL), 1000),
    ("ragged_72x40x20_clustered", rep(I.CFG_CLUSTERED, n=(72, 40, 20), n_particles=3000,
                                       cluster_std=0.3), 3000),
    ("small_16x12x10_sigma1.5", rep(I.CFG_CLUSTERED, n=(16, 12, 10), L=(2 * math.pi, 5.0, 4.0),
                                     n_particles=500, cluster_std=0.5, kmax=3.0), 500),
    ("aniso_96x33x17", rep(I.CFG_SMALL, n=(96, 33, 17), L=(2 * math.pi, 2.0, 1.0)), 2000),
    # isotropic spacing where r_c / dx rounds to just below 3 (windows of 5-7
    # nodes), two x-tiles of 64 and 8 nodes
    ("iso_72x40x20", rep(I.CFG_SMALL, n=(72, 40, 20), kmax=3.0,
                         L=(2 * math.pi, 2 * math.pi * 40 / 72, 2 * math.pi * 20 / 72)), 3000),
    # y spacing a third of x: y-windows of 19 nodes, beyond the x/y-halo tiles
    # (the kernels cut pieces in y and z instead)
    ("fine_y_32x96x24", rep(I.CFG_SMALL, n=(32, 96, 24), kmax=3.0), 1500),
    # large enough for tiles whose staged box needs no periodic wrap (staged
    # by one TMA copy) next to wrapping ones
    ("tma_256x64x16", rep(I.CFG_SMALL, n=(256, 64, 16), kmax=3.0,
                          L=(2 * math.pi, 2 * math.pi * 64 / 256, 2 * math.pi * 16 / 256)),
     20000),
    # rows of an odd number of nodes: no 16-byte row alignment, so the tile
    # kernels stage and write out word by word
    # sigma_R = 1.5 dx: x-tiles of 34 nodes (the second starts off a 16-byte
    # boundary and is staged word by word, the first by bulk row copies)
    ("split_x_68x24x20_sigma1.5", rep(I.CFG_CLUSTERED, n=(68, 24, 20), n_particles=2000,
                                      cluster_std=0.3, kmax=3.0,
                                      L=(2 * math.pi, 2 * math.pi * 24 / 68,
                                         2 * math.pi * 20 / 68)), 2000),
    ("odd_x_45x30x20", rep(I.CFG_SMALL, n=(45, 30, 20), kmax=3.0,
                           L=(2 * math.pi, 2 * math.pi * 30 / 45, 2 * math.pi * 20 / 45)), 1500),
    # sigma_R = 1.5 dx on 24^3: y-tiles of 16 and 8 rows against a halo 9
    # rows deep, so rows of the thin tile are rims on both sides
    ("thin_y_tile_24cube_sigma1.5", rep(I.CFG_CLUSTERED, n=(24, 24, 24), n_particles=600,
                                        n_clusters=5, cluster_std=0.4, kmax=3.0), 600),
    # sigma_R = 2.5 dx: windows of 15-16 nodes, the widest the FP32 x/y-halo
    # tiles take (16 x-weights per particle)
    ("wide_80x48x40_sigma2.5", rep(I.CFG_SMALL, n=(80, 48, 40), kmax=3.0, sigma_over_dx=2.5,
                                   L=(2 * math.pi, 2 * math.pi * 48 / 80,
                                      2 * math.pi * 40 / 80)), 600),
]


def _setup(w, npart):
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field if npart <= 3000 else None, n_particles=npart)
    return grid, st


def _near_window_ends(p, w):
    """Positions whose x N/L lies within a few units in the last place of
    j + c' or j - c' (a window end changes there) or of a node j (the home
    cell and the fractional position change), on each axis; -0.0 too."""
    L = np.array(w.L, dtype=np.float64)
    n = np.array(w.n, dtype=np.float64)
    sig = np.sqrt(2.0 * p["nu"] * p["eps_R"])
    cp = p["cutoff"] * sig * n / L
    cols = []
    for j in (3, 5, 11):
        for centre in (j + cp, j - cp, np.full(3, float(j))):
            x0 = np.mod(centre, n) * (L / n)
            for k in range(-3, 4):
                x = x0.copy()
                for _ in range(abs(k)):
                    x = np.nextafter(x, np.inf if k > 0 else 0.0)
                cols.append(np.clip(x, 0.0, np.nextafter(L, 0)))
    cols.append(np.array([-0.0, -0.0, -0.0]))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_windows_bit_exact(erpp, oracle_lib, name, w, npart):
    """Integer stencil membership is identical to the oracle's."""
    p = w.params()
    _, st = _setup(w, npart)
    # add particles on nodes, on cell faces and next to the box edges
    L = np.array(w.L)[:, None]
    n = np.array(w.n)[:, None]
    special = np.concatenate([
        (np.arange(12) % n) * (L / n),
        (np.arange(12) % n + 0.5) * (L / n),
        np.nextafter(L, 0) * np.ones((3, 4)),
        np.zeros((3, 2)),
        _near_window_ends(p, w),
    ], axis=1)
    x = np.concatenate([st.x, special], axis=1)
    ctx = erpp.Context(p, precision="fp32")
    lo, hi = ctx.debug_windows(cuda(x))
    rlo, rhi = oracle_lib.windows(p, x)
    np.testing.assert_array_equal(lo.cpu().numpy(), rlo)
    np.testing.assert_array_equal(hi.cpu().numpy(), rhi)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_scatter_source(erpp, oracle_lib, precision, name, w, npart):
    p = w.params()
    _, st = _setup(w, npart)
    D = I.make_forces(npart, 1.0, seed=7)
    ctx = erpp.Context(p, precision=precision)
    S = ctx.scatter_source(cuda(st.x), cuda(D))
    ctx.check()
    ref = oracle_lib.scatter(p, st.x, D)
    assert rel(S.cpu().numpy(), ref) < TOL[precision]


@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_scatter_reproducible(erpp, name, w, npart):
    """Repeated FP32 scatters of the same cloud are bit-identical: pieces land
    in their tiles in a different order each time, but the fixed-point sums do
    not depend on it and every halo node is merged in a fixed order, whichever
    block merges it."""
    import torch
    p = w.params()
    _, st = _setup(w, npart)
    D = I.make_forces(npart, 1.0, seed=11)
    ctx = erpp.Context(p, precision="fp32")
    x, Dt = cuda(st.x), cuda(D)
    S1 = ctx.scatter_source(x, Dt).clone()
    for _ in range(3):
        S2 = ctx.scatter_source(x, Dt)
        ctx.check()
        assert torch.equal(S1, S2)


@pytest.mark.parametrize("kahan", [False, True])
@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_scatter_modes(erpp, oracle_lib, kahan, name, w, npart):
    """The ways the FP32 scatter handles tile halos (strips and two merge
    kernels; the x-halo through thread-block clusters; x-windows cut at
    x-tile boundaries, y-halo through strips): each matches the oracle and
    each is reproducible bit for bit."""
    import torch
    p = w.params()
    _, st = _setup(w, npart)
    D = I.make_forces(npart, 1.0, seed=13)
    ref = oracle_lib.scatter(p, st.x, D)
    x, Dt = cuda(st.x), cuda(D)
    out = {}
    for mode in ("merge", "cluster", "xclip"):
        ctx = erpp.Context(p, precision="fp32", kahan=kahan)
        ctx.set_scatter_mode(mode)
        S1 = ctx.scatter_source(x, Dt).clone()
        S2 = ctx.scatter_source(x, Dt)
        ctx.check()
        if not kahan:
            assert torch.equal(S1, S2), mode
        assert rel(S1.cpu().numpy(), ref) < TOL["fp32"], mode
        out[mode] = S1.cpu().numpy()
        ctx.close()
    # the same pieces and scales: only the order of the halo additions differs
    # (cut windows change each tile's pieces and fixed-point scale, so the
    # cut form is held to the oracle only)
    assert rel(out["cluster"], out["merge"]) < 1e-6


@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_step_xclip(erpp, oracle_lib, name, w, npart):
    """The coupling step with x-windows cut at x-tile boundaries (gather and
    scatter on the cut pieces) against the oracle."""
    p = w.params(gravity=(0.0, -9.81, 0.0))
    grid, st = _setup(w, npart)
    ctx = erpp.Context(p, precision="fp32")
    ctx.set_scatter_mode("xclip")
    ps = erpp.ParticleState.from_numpy(st)
    S = ctx.step(grid_t(grid, "fp32"), ps, first_step=False)
    ctx.check()
    ref = st.copy()
    S_ref = oracle_lib.step(p, grid, ref, first_step=False)
    assert rel(S.cpu().numpy(), S_ref) < TOL["fp32"]
    assert rel(ps.D.cpu().numpy(), ref.D) < TOL["fp32"]
    assert rel(ps.v.cpu().numpy(), ref.v) < TOL["fp32"]


@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_step_reproducible(erpp, name, w, npart):
    """The whole FP32 step on x/y-halo tiles is reproducible bit for bit: the
    gather keeps every unit's sums in a slot of its own and adds them in a
    fixed order (planes, then pieces), a unit's rows are summed in the same
    order wherever its walk starts, and the scatter's fixed-point sums and
    tile scale do not depend on the order of the pieces.  (The x-halo tiles
    of windows longer than 16 nodes in y gather with FP32 atomics.)"""
    import torch
    p = w.params()
    grid, st = _setup(w, npart)
    ctx = erpp.Context(p, precision="fp32")
    if ctx.tiling()[0] != 4:
        pytest.skip("x-halo tiles: FP32 atomics in the gather")
    u = grid_t(grid, "fp32")
    out = []
    for _ in range(2):
        ps = erpp.ParticleState.from_numpy(st)
        S = ctx.step(u, ps, first_step=False)
        ctx.check()
        out.append((S.clone(), ps.D.clone(), ps.v.clone(), ps.x.clone()))
    for a, b in zip(*out):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_launch_count(erpp, precision):
    """The library's own count of the kernels one step launches: FP32 =
    binning (count, one scan kernel for boxes of at most 65536 tiles, fill)
    + gather + advance + scatter + one or two halo merge kernels; FP64 plain
    form = gather + advance + scatter."""
    w = CASES[0][1]
    grid, st = _setup(w, CASES[0][2])
    ctx = erpp.Context(w.params(), precision=precision)
    assert ctx.last_step_launches() == 0
    ps = erpp.ParticleState.from_numpy(st)
    ctx.step(grid_t(grid, precision), ps, first_step=True)
    ctx.check()
    n = ctx.last_step_launches()
    if precision == "fp64":
        assert n == 3
    else:
        # binning 3, gather, advance, scatter, then the halo merges: two
        # through strips (8), one with the x-halo in clusters (7)
        assert n == 8
        for mode, want in (("cluster", 7), ("xclip", 7), ("merge", 8)):
            ctx.set_scatter_mode(mode)
            ctx.step(grid_t(grid, precision), ps)
            ctx.check()
            assert ctx.last_step_launches() == want, mode


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_interpolate(erpp, oracle_lib, precision, name, w, npart):
    p = w.params()
    grid, st = _setup(w, npart)
    ctx = erpp.Context(p, precision=precision)
    up = ctx.interpolate(grid_t(grid, precision), cuda(st.x))
    ctx.check()
    ref = oracle_lib.gather(p, st.x, grid)
    assert rel(up.cpu().numpy(), ref) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("self_removal", [True, False])
@pytest.mark.parametrize("name,w,npart", CASES, ids=[c[0] for c in CASES])
def test_step(erpp, oracle_lib, precision, self_removal, name, w, npart):
    p = w.params(gravity=(0.0, -9.81, 0.0))
    grid, st = _setup(w, npart)
    ctx = erpp.Context(p, precision=precision, self_removal=self_removal)
    ps = erpp.ParticleState.from_numpy(st)
    S = ctx.step(grid_t(grid, precision), ps, first_step=False)
    ctx.check()
    ref = st.copy()
    S_ref = oracle_lib.step(dict(p, self_removal=self_removal), grid, ref, first_step=False)
    tol = TOL[precision]
    assert rel(S.cpu().numpy(), S_ref) < tol
    assert rel(ps.D.cpu().numpy(), ref.D) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol
    np.testing.assert_array_equal(ps.x_prev.cpu().numpy(), st.x)
    # positions: FP64 integration of FP64 (or FP32-accurate) velocities
    dxp = np.abs(ps.x.cpu().numpy() - ref.x)
    dxp = np.minimum(dxp, np.array(w.L)[:, None] - dxp)
    assert dxp.max() < (1e-15 if precision == "fp64" else 1e-12) * 10 * max(w.L)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_particle_advance_standalone(erpp, oracle_lib, precision):
    w = I.CFG_SMALL
    p = w.params(gravity=(0.0, 0.0, -1.0))
    grid, st = _setup(w, 1000)
    up = oracle_lib.gather(p, st.x, grid)
    ctx = erpp.Context(p, precision=precision)
    ps = erpp.ParticleState.from_numpy(st)
    ctx.particle_advance(cuda(up), ps, first_step=False)
    ref = st.copy()
    oracle_lib.advance(p, up, ref, first_step=False)
    tol = 1e-6 if precision == "fp32" else 1e-13
    assert rel(ps.D.cpu().numpy(), ref.D) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_clustered_ten_steps(erpp, oracle_lib, precision):
    """The clustered workload (50 Gaussian clusters, std 0.05, mean shear
    S = 1, sigma_R = 1.5 dx) on a reduced grid: ten coupled steps with the
    fluid frozen, FP32 and FP64 against the FP64 oracle."""
    w = rep(I.CFG_CLUSTERED, n=(64, 64, 64), n_particles=20000)
    p = w.params()
    grid, st = _setup(w, 20000)
    ctx = erpp.Context(p, precision=precision)
    ps = erpp.ParticleState.from_numpy(st)
    u = grid_t(grid, precision)
    ref = st.copy()
    for k in range(10):
        S = ctx.step(u, ps, first_step=(k == 0))
        S_ref = oracle_lib.step(p, grid, ref, first_step=(k == 0))
    ctx.check()
    tol = TOL[precision]
    assert rel(S.cpu().numpy(), S_ref) < tol
    assert rel(ps.D.cpu().numpy(), ref.D) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol


@pytest.mark.parametrize("mode", ["fp32", "fp32_kahan", "fp64"])
def test_clustered_full_size_error_report(erpp, oracle_lib, mode):
    """The clustered FP32-versus-FP64 workload at full size: 128^3, 100k
    particles in 50 clusters, sigma_R = 1.5 dx, mean shear 1, ten coupled
    steps with the fluid frozen.  Prints the relative L2 error of every result
    (source, forces, velocities, positions) against the FP64 oracle and holds
    it to the tolerance of one step times the number of steps (errors
    compound through the particle state)."""
    w = I.CFG_CLUSTERED
    p = w.params()
    grid, st = _setup(w, w.n_particles)
    precision = "fp64" if mode == "fp64" else "fp32"
    ctx = erpp.Context(p, precision=precision, kahan=(mode == "fp32_kahan"))
    ps = erpp.ParticleState.from_numpy(st)
    u = grid_t(grid, precision)
    ref = st.copy()
    for k in range(10):
        S = ctx.step(u, ps, first_step=(k == 0))
        S_ref = oracle_lib.step(p, grid, ref, first_step=(k == 0))
    ctx.check()
    errs = {"S": rel(S.cpu().numpy(), S_ref), "D": rel(ps.D.cpu().numpy(), ref.D),
            "v": rel(ps.v.cpu().numpy(), ref.v)}
    dxp = np.abs(ps.x.cpu().numpy() - ref.x)
    dxp = np.minimum(dxp, np.array(w.L)[:, None] - dxp)
    errs["x_max_abs"] = float(dxp.max())
    print(f"\nclustered 128^3 / 100k, 10 steps, {mode}: " +
          ", ".join(f"{k} {v:.3e}" for k, v in errs.items()))
    tol = 10 * TOL[precision]
    assert errs["S"] < tol and errs["D"] < tol and errs["v"] < tol
    # positions integrate the velocities in FP64: over the ten steps their
    # error is at most steps * dt * (velocity tolerance) * max |v|
    # (FP64: a few ulps of the coordinates)
    vmax = float(np.abs(ref.v).max())
    assert errs["x_max_abs"] < max(10 * p["dt"] * TOL[precision] * vmax, 1e-12)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_momentum_conservation(erpp, oracle_lib, precision):
    w = rep(I.CFG_CLUSTERED, n=(72, 40, 20))
    p = w.params()
    _, st = _setup(w, 3000)
    ctx = erpp.Context(p, precision=precision)
    x, D = cuda(st.x), cuda(st.D)
    S = ctx.scatter_source(x, D)
    Pg, Pp = ctx.momentum(S, x, D)
    rg, rp = oracle_lib.momentum(p, st.x, st.D, oracle_lib.scatter(p, st.x, st.D))
    scale = np.abs(rp).max()
    np.testing.assert_allclose(Pp, rp, rtol=1e-12, atol=1e-13 * scale)
    np.testing.assert_allclose(Pg, rg, atol=(1e-6 if precision == "fp32" else 1e-12) * scale)


def test_kahan_scatter(erpp, oracle_lib):
    """Compensated FP32 accumulation on a dense cluster (thousands of
    contributions per node) is closer to the FP64 oracle than plain FP32."""
    w = rep(I.CFG_CLUSTERED, n=(48, 48, 48), n_clusters=2, cluster_std=0.02)
    p = w.params()
    _, st = _setup(w, 20000)
    D = I.make_forces(20000, 1.0, seed=3) + 0.5
    ref = oracle_lib.scatter(p, st.x, D)
    errs = {}
    for kahan in (False, True):
        ctx = erpp.Context(p, precision="fp32", kahan=kahan)
        S = ctx.scatter_source(cuda(st.x), cuda(D))
        errs[kahan] = rel(S.cpu().numpy(), ref)
    assert errs[True] < TOL["fp32"] and errs[False] < TOL["fp32"]
    assert errs[True] <= errs[False]


def test_permutation_invariance(erpp):
    w = rep(I.CFG_CLUSTERED, n=(72, 40, 20))
    p = w.params()
    _, st = _setup(w, 3000)
    perm = np.random.default_rng(1).permutation(3000)
    ctx = erpp.Context(p, precision="fp32")
    S1 = ctx.scatter_source(cuda(st.x), cuda(st.D)).cpu().numpy()
    S2 = ctx.scatter_source(cuda(st.x[:, perm]), cuda(st.D[:, perm])).cpu().numpy()
    assert rel(S2, S1) < 1e-6


def test_edge_cases(erpp, oracle_lib):
    import torch
    w = rep(I.CFG_SMALL, n=(40, 24, 20))
    p = w.params()
    ctx = erpp.Context(p, precision="fp32")
    # no particles: the source is zero everywhere (fully overwritten)
    S = ctx.new_grid().fill_(7.0)
    ctx.scatter_source(cuda(np.zeros((3, 0))), cuda(np.zeros((3, 0))), S=S)
    assert float(S.abs().max()) == 0.0
    # one particle at the origin and one just below L (windows wrap)
    L = np.array(w.L)
    x = np.stack([np.zeros(3), np.nextafter(L, 0)], axis=1)
    D = np.array([[1.0, -2.0], [0.5, 0.25], [-1.0, 3.0]])
    S = ctx.scatter_source(cuda(x), cuda(D))
    assert rel(S.cpu().numpy(), oracle_lib.scatter(p, x, D)) < TOL["fp32"]
    # all particles in one cell (heavy atomic contention)
    xc = np.full((3, 4000), 1.0) + 1e-3 * np.random.default_rng(0).random((3, 4000))
    Dc = np.random.default_rng(1).standard_normal((3, 4000))
    S = ctx.scatter_source(cuda(xc), cuda(Dc))
    assert rel(S.cpu().numpy(), oracle_lib.scatter(p, xc, Dc)) < TOL["fp32"]
    # invalid positions are reported, never trapped
    bad = x.copy()
    bad[0, 0] = float("nan")
    bad[1, 1] = L[1]
    ctx.scatter_source(cuda(bad), cuda(D))
    with pytest.raises(erpp.ErppError) as ei:
        ctx.check()
    assert ei.value.status == 4  # ERPP_ERANGE
    ctx.check()  # the error word was cleared
    torch.cuda.synchronize()


def test_invalid_arguments(erpp):
    p = I.CFG_SMALL.params()
    with pytest.raises(erpp.ErppError):
        erpp.Context(dict(p, cutoff=40.0))  # 2 r_c >= L
    with pytest.raises(erpp.ErppError):
        erpp.Context(dict(p, nu=-1.0))
    with pytest.raises(erpp.ErppError):
        erpp.Context(p, precision="fp64", kahan=True)


def test_widest_window_fp64(erpp, oracle_lib):
    """sigma_R = 5 dx at cutoff 3: windows of 30-31 nodes, the widest the
    library takes.  The FP64 plain form matches the oracle; an FP32 context refuses the
    parameters (its tiles take x-windows of at most 16 nodes)."""
    from paper_1405_6969_gb300 import ErppError
    w = rep(I.CFG_SMALL, n=(72, 64, 64), kmax=3.0, sigma_over_dx=5.0,
            L=(2 * math.pi * 72 / 64, 2 * math.pi, 2 * math.pi))
    p = w.params()
    grid, st = _setup(w, 200)
    # windows of 30 nodes, 31 for a particle whose s = x N / L is an integer
    lo, hi = oracle_lib.windows(p, st.x)
    assert (hi - lo + 1).max() >= 30
    ctx = erpp.Context(p, precision="fp64")
    S = ctx.scatter_source(cuda(st.x), cuda(st.D))
    assert rel(S.cpu().numpy(), oracle_lib.scatter(p, st.x, st.D)) < 1e-12
    up = ctx.interpolate(grid_t(grid, "fp64"), cuda(st.x)).cpu().numpy()
    ref = oracle_lib.gather(p, st.x, grid)
    assert np.abs(up - ref).max() < 1e-12 * np.abs(ref).max()
    ctx.check()
    with pytest.raises(ErppError):
        erpp.Context(p, precision="fp32")

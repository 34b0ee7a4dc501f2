"""GPU parity of the batched step (erpp_batch_* through the binding).

Each box of a heterogeneous batch (different grids, particle counts and
parameters) must match the FP64 oracle's step of that box alone, within the
step tolerances (relative L2: 1e-5 FP32, 1e-12 FP64), whether the batch runs
as one replayed CUDA graph or as plain launches box after box.
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


def small_boxes():
    """Six boxes: cubic and anisotropic grids, sigma_R = dx and 1.5 dx,
    uniform and clustered clouds, with and without shear and gravity."""
    b = []
    for i, (n, L, npart, sig, cloud, shear, grav) in enumerate([
        ((32, 32, 32), (2 * math.pi,) * 3, 1000, 1.0, "uniform", 0.0, 0.0),
        ((48, 40, 24), (2 * math.pi, 5.0, 3.0), 3000, 1.0, "uniform", 1.0, -9.81),
        ((24, 24, 24), (2 * math.pi,) * 3, 200, 1.5, "clusters", 0.0, 0.0),
        ((72, 40, 20), (2 * math.pi, 2 * math.pi * 40 / 72, 2 * math.pi * 20 / 72), 2500, 1.0,
         "clusters", 0.5, 0.0),
        ((40, 40, 40), (2 * math.pi,) * 3, 1, 1.0, "uniform", 0.0, -1.0),
        ((64, 32, 32), (4 * math.pi, 2 * math.pi, 2 * math.pi), 4000, 1.5, "uniform", 1.0, 0.0),
    ]):
        w = I.Workload(name=f"b{i}", n=n, L=L, n_particles=npart, sigma_over_dx=sig,
                       kmax=3.0, field_seed=i, particle_seed=i, cloud=cloud, n_clusters=5,
                       cluster_std=0.4, shear_rate=shear, gravity=(0.0, grav, 0.0))
        b.append(w)
    return b


def _build(erpp, precision, boxes):
    import torch
    dtype = torch.float32 if precision == "fp32" else torch.float64
    entries, refs = [], []
    for w in boxes:
        grid, field = I.make_grid(w)
        st = I.make_particles(w, field)
        u = cuda(grid, dtype)
        S = torch.empty_like(u)
        ps = erpp.ParticleState.from_numpy(st)
        entries.append((w.params(), u, ps, S))
        refs.append((grid, st.copy()))
    return entries, refs


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_step_matches_oracle(erpp, oracle_lib, precision, use_graph):
    boxes = small_boxes()
    entries, refs = _build(erpp, precision, boxes)
    batch = erpp.Batch(entries, precision=precision)
    for k in range(2):
        batch.step(first_step=(k == 0), use_graph=use_graph)
        for (p, _, _, _), (grid, ref) in zip(entries, refs):
            oracle_lib.step(p, grid, ref, first_step=(k == 0))
    batch.check()
    tilings = [batch.tiling(i) for i in range(len(boxes))]
    assert all(t[0] in (3, 4) for t in tilings)
    tol = TOL[precision]
    for (p, u, ps, S), (grid, ref), w in zip(entries, refs, boxes):
        S_ref = oracle_lib.scatter(p, ref.x_prev, ref.D)
        assert rel(S.cpu().numpy(), S_ref) < tol, w.name
        assert rel(ps.D.cpu().numpy(), ref.D) < tol, w.name
        assert rel(ps.v.cpu().numpy(), ref.v) < tol, w.name
        dxp = np.abs(ps.x.cpu().numpy() - ref.x)
        dxp = np.minimum(dxp, np.array(w.L)[:, None] - dxp)
        assert dxp.max() < 1e-10 * max(w.L), w.name
    batch.close()


def same_variant_boxes():
    """Five boxes whose stencils share one window length (sigma_R = dx along
    x): the graph runs the step of all of them as nine multi-box launches.
    Cubic, anisotropic and ragged grids, dense and sparse clouds, one box
    with a single particle."""
    b = []
    for i, (n, L, npart, cloud, shear) in enumerate([
        ((64, 64, 64), (2 * math.pi,) * 3, 20000, "uniform", 1.0),
        ((72, 40, 20), (2 * math.pi, 2 * math.pi * 40 / 72, 2 * math.pi * 20 / 72), 2500,
         "clusters", 0.5),
        ((96, 48, 48), (2 * math.pi, math.pi, math.pi), 6000, "uniform", 0.0),
        ((40, 40, 40), (2 * math.pi,) * 3, 1, "uniform", 0.0),
        ((130, 34, 18), (2 * math.pi, 2 * math.pi * 34 / 130, 2 * math.pi * 18 / 130), 3000,
         "clusters", 0.0),
    ]):
        b.append(I.Workload(name=f"m{i}", n=n, L=L, n_particles=npart, sigma_over_dx=1.0,
                            kmax=3.0, field_seed=10 + i, particle_seed=10 + i, cloud=cloud,
                            n_clusters=4, cluster_std=0.5, shear_rate=shear))
    return b


def test_multi_box_launches_match_oracle_and_plain_launches(erpp, oracle_lib):
    """The multi-box graph (binning, advance and merges over every box's
    particles and tiles, persistent gather and scatter pulling (box, tile)
    items) against the oracle per box, over three steps, and bit for bit
    against the same batch run as plain launches box after box."""
    boxes = same_variant_boxes()
    entries, refs = _build(erpp, "fp32", boxes)
    entries2, _ = _build(erpp, "fp32", boxes)
    batch = erpp.Batch(entries, precision="fp32")
    batch.set_form("multi")
    plain = erpp.Batch(entries2, precision="fp32")
    for k in range(3):
        batch.step(first_step=(k == 0), use_graph=True)
        plain.step(first_step=(k == 0), use_graph=False)
        for (p, _, _, _), (grid, ref) in zip(entries, refs):
            oracle_lib.step(p, grid, ref, first_step=(k == 0))
    batch.check()
    plain.check()
    assert all(batch.tiling(i)[0] == 4 for i in range(len(boxes)))
    # all boxes together: clear, count, scan, fill, gather, advance, scatter,
    # two merges
    assert batch.last_step_launches() == 9
    for (p, u, ps, S), (_, u2, ps2, S2), (grid, ref), w in zip(entries, entries2, refs, boxes):
        S_ref = oracle_lib.scatter(p, ref.x_prev, ref.D)
        assert rel(S.cpu().numpy(), S_ref) < 1e-5, w.name
        assert rel(ps.D.cpu().numpy(), ref.D) < 1e-5, w.name
        assert rel(ps.v.cpu().numpy(), ref.v) < 1e-5, w.name
        # the same kernels' arithmetic on the same data: bit for bit
        assert np.array_equal(S.cpu().numpy(), S2.cpu().numpy()), w.name
        assert np.array_equal(ps.D.cpu().numpy(), ps2.D.cpu().numpy()), w.name
        assert np.array_equal(ps.x.cpu().numpy(), ps2.x.cpu().numpy()), w.name
    batch.close()
    plain.close()


def test_graph_replay_sees_new_contents(erpp, oracle_lib):
    """The graph keeps addresses, not values: rewriting a box's field and
    particles in place between replays is reflected in the next step."""
    boxes = small_boxes()[:3]
    entries, refs = _build(erpp, "fp32", boxes)
    batch = erpp.Batch(entries, precision="fp32")
    batch.step(first_step=True)
    # new field and a fresh cloud for box 1, written into the same buffers
    w = dataclasses.replace(boxes[1], field_seed=77, particle_seed=78)
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    p, u, ps, S = entries[1]
    u.copy_(cuda(grid, u.dtype))
    for name in ("x", "v", "x_prev", "D"):
        getattr(ps, name).copy_(cuda(getattr(st, name)))
    batch.step(first_step=True)
    batch.check()
    ref = st.copy()
    S_ref = oracle_lib.step(p, grid, ref, first_step=True)
    assert rel(S.cpu().numpy(), S_ref) < 1e-5
    assert rel(ps.D.cpu().numpy(), ref.D) < 1e-5
    batch.close()


def test_batch_rejects_bad_descriptors(erpp):
    import torch
    w = small_boxes()[0]
    grid, field = I.make_grid(w)
    u = cuda(grid, torch.float32)
    ps = erpp.ParticleState.from_numpy(I.make_particles(w, field))
    with pytest.raises(ValueError):
        erpp.Batch([(w.params(), u, ps, torch.empty((3, 4, 4, 4), device="cuda"))])
    bad = dict(w.params(), cutoff=40.0)  # 2 r_c beyond the box
    with pytest.raises(erpp.ErppError):
        erpp.Batch([(bad, u, ps, torch.empty_like(u))])


def test_batch_autotune_keeps_results(erpp, oracle_lib, tmp_path):
    """Per-box tile shapes chosen by the autotuner (graphs captured again
    afterwards) give the same results as the oracle."""
    boxes = small_boxes()
    entries, refs = _build(erpp, "fp32", boxes)
    batch = erpp.Batch(entries, precision="fp32")
    batch.step(first_step=True)            # a graph captured with default tiles
    chosen = batch.autotune(steps=1, warmup=1, cache_path=str(tmp_path / "t.json"))
    assert len(chosen) == len(boxes)
    batch.step(first_step=True)            # captured again with the new tiles
    batch.step(first_step=False)
    batch.check()                          # replays ran without device errors
    batch.close()
    # a fresh batch with the chosen shapes against the oracle, two steps
    entries, refs = _build(erpp, "fp32", boxes)
    batch = erpp.Batch(entries, precision="fp32")
    for i, t in enumerate(chosen):
        if t is not None:
            batch.set_tiling(i, *t)
    for k in range(2):
        batch.step(first_step=(k == 0))
        for (p, _, _, _), (grid, ref) in zip(entries, refs):
            oracle_lib.step(p, grid, ref, first_step=(k == 0))
    batch.check()
    for (p, u, ps, S), (grid, ref), w in zip(entries, refs, boxes):
        S_ref = oracle_lib.scatter(p, ref.x_prev, ref.D)
        assert rel(S.cpu().numpy(), S_ref) < 1e-5, w.name
        assert rel(ps.D.cpu().numpy(), ref.D) < 1e-5, w.name
    batch.close()

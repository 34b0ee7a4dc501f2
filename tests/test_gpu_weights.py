"""GPU parity of the other weights (ERPP_PIC, ERPP_POINT_GATHER) against the
oracle (oracle/weights.py), and the paper's PIC comparison on the GPU.

* PIC source, PIC and point-value gathers, and three coupling steps with each,
  on several grids (cubic, ragged, odd sizes; particles on the lower and
  next to the upper faces; one particle; none): relative L2 within 1e-5 in
  FP32 (the PIC source adds with device atomics: FP32 sums in arrival
  order), 1e-12 in FP64; gathered velocities 1e-5 / 1e-12 of their scale;
* the full 512 x 256 x 256 grid with 1M particles: the PIC source on the
  whole grid, the gathers on a sample of particles;
* the momentum of the PIC source equals the particles' (unit-mass weights);
* the flags that cannot combine are refused;
* coupled settling (Sec. 3.2.2, the PIC panels of Figs. velo_vs_t and
  velo_terminal): the PIC particle misses its terminal velocity by more than
  twice the ERPP particle at every d_p/Dx, and its error falls as d_p/Dx -> 0.
"""

import dataclasses
import json
import math
import os

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "settling_coupled.json")))


@pytest.fixture(scope="module")
def erpp(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_6969_gb300 as pkg
    return pkg


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _dtype(precision):
    import torch
    return torch.float32 if precision == "fp32" else torch.float64


def _tol(precision):
    return 1e-5 if precision == "fp32" else 1e-12


def _case(name):
    """(params, state, grid field) of one parity case."""
    if name == "small_32":
        w = I.CFG_SMALL
    elif name == "ragged_45x30x20":
        w = I.CFG_SMALL.scaled("ragged", (45, 30, 20), 800,
                               L=(2 * math.pi * 45 / 32, 2 * math.pi * 30 / 32,
                                  2 * math.pi * 20 / 32))
    else:
        w = I.CFG_SMALL.scaled("odd", (27, 33, 25), 600,
                               L=(2 * math.pi * 27 / 32, 2 * math.pi * 33 / 32,
                                  2 * math.pi * 25 / 32))
    w = dataclasses.replace(w, shear_rate=0.7)
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    # particles on the lower faces and just below the upper ones
    st.x[:, 0] = 0.0
    for a in range(3):
        st.x[a, 1] = np.nextafter(w.L[a], 0.0)
    st.x[:, 2] = [np.nextafter(w.L[0], 0.0), 0.0, w.L[2] / 2]
    return w, st, grid


CASES = ["small_32", "ragged_45x30x20", "odd_27x33x25"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", CASES)
def test_pic_scatter_matches_oracle(erpp, oracle_lib, precision, case):
    from oracle import weights as W
    w, st, _ = _case(case)
    p = w.params()
    ctx = erpp.Context(p, precision=precision, weights="pic")
    S = ctx.scatter_source(cuda(st.x), cuda(st.D))
    ref = W.pic_scatter(p, st.x, st.D)
    assert rel(S.cpu().numpy(), ref) < _tol(precision)
    # one particle, and none (the source is zeroed)
    S1 = ctx.scatter_source(cuda(st.x[:, 5:6]), cuda(st.D[:, 5:6]))
    assert rel(S1.cpu().numpy(), W.pic_scatter(p, st.x[:, 5:6], st.D[:, 5:6])) < _tol(precision)
    S0 = ctx.scatter_source(cuda(np.zeros((3, 0))), cuda(np.zeros((3, 0))), S=S1)
    assert float(S0.abs().max()) == 0.0
    ctx.check()
    # momentum: dV sum S = -(1/rho_f) sum D (trilinear weights carry unit mass)
    grid_m, part_m = ctx.momentum(S, cuda(st.x), cuda(st.D))
    np.testing.assert_allclose(grid_m, part_m, rtol=0,
                               atol=10 * _tol(precision) * np.abs(part_m).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["pic", "point"])
@pytest.mark.parametrize("case", CASES)
def test_gathers_match_oracle(erpp, oracle_lib, precision, kind, case):
    from oracle import weights as W
    w, st, grid = _case(case)
    p = w.params()
    ctx = erpp.Context(p, precision=precision, weights=kind)
    up = ctx.interpolate(cuda(grid, _dtype(precision)), cuda(st.x)).cpu().numpy()
    ref = W.pic_gather(p, st.x, grid) if kind == "pic" else W.point_gather(p, st.x, grid)
    assert np.abs(up - ref).max() < _tol(precision) * np.abs(ref).max()
    ctx.check()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["pic", "point"])
def test_steps_match_oracle(erpp, oracle_lib, precision, kind):
    from oracle import weights as W
    w, st, grid = _case("ragged_45x30x20")
    p = w.params(gravity=(0.0, -1.5, 0.4))
    ctx = erpp.Context(p, precision=precision, weights=kind)
    ps = erpp.ParticleState.from_numpy(st)
    u = cuda(grid, _dtype(precision))
    S = ctx.new_grid()
    ref = st.copy()
    for k in range(3):
        ctx.step(u, ps, S=S, first_step=(k == 0))
        S_ref = W.step(p, grid, ref, kind, first_step=(k == 0))
        tol = _tol(precision)
        assert rel(S.cpu().numpy(), S_ref) < tol, k
        for name in ("v", "D"):
            assert rel(getattr(ps, name).cpu().numpy(), getattr(ref, name)) < tol, (k, name)
        for name in ("x", "x_prev"):
            got = getattr(ps, name).cpu().numpy()
            assert np.abs(got - getattr(ref, name)).max() < 1e-9, (k, name)
    ctx.check()
    assert ctx.last_step_launches() >= 3


def test_full_size_sampled(erpp, oracle_lib):
    """512 x 256 x 256, 1M particles (the benchmark's grid and cloud), FP32:
    the PIC source on the whole grid; both gathers on 2000 sampled particles."""
    import torch
    from oracle import weights as W
    w = I.CFG_SHEAR
    p = w.params()
    st = I.make_particles(w, None)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, w.n[2], w.n[1], w.n[0])).astype(np.float32)
    ut = cuda(u, torch.float32)
    xs, Ds = cuda(st.x), cuda(st.D)
    pic = erpp.Context(p, precision="fp32", weights="pic")
    S = pic.scatter_source(xs, Ds)
    ref = W.pic_scatter(p, st.x, st.D)
    assert rel(S.cpu().numpy(), ref) < 1e-5
    del S, ref
    idx = rng.choice(w.n_particles, 2000, replace=False)
    for kind, fn in (("pic", W.pic_gather), ("point", W.point_gather)):
        ctx = pic if kind == "pic" else erpp.Context(p, precision="fp32", weights="point")
        up = ctx.interpolate(ut, xs).cpu().numpy()[:, idx]
        r = fn(p, st.x[:, idx], u.astype(np.float64))
        assert np.abs(up - r).max() < 1e-5 * np.abs(r).max(), kind
        ctx.check()


def test_refused_combinations(erpp):
    from paper_1405_6969_gb300 import ErppError
    w = I.CFG_SMALL
    p = w.params()
    with pytest.raises(ErppError):
        erpp.Context(p, precision="fp32", weights="pic", kahan=True)
    ctx = erpp.Context(p, precision="fp64", weights="pic")
    st = I.make_particles(w, None)
    with pytest.raises(ErppError):
        ctx.scatter_backward(cuda(st.x), cuda(st.D), ctx.new_grid().zero_())


def _settle(erpp, dp_over_dx, weights, N=24):
    """One heavy particle settling from rest, two-way coupled through the
    fluid stand-in (the set-up of the ERPP settling test, sigma_R = dx)."""
    import torch
    L = GOLD["box_length"]
    nu, rho_ratio = 0.1, 1000.0
    dx = L / N
    d = dp_over_dx * dx
    tau = rho_ratio * d * d / (18 * nu)
    vt = 1e-3
    g = vt / tau / (1 - 1 / rho_ratio)
    dt = tau / 20
    p = dict(n=(N, N, N), L=(L, L, L), nu=nu, rho_f=1.0, eps_R=dx ** 2 / (2 * nu),
             cutoff=3.0, dt=dt, gravity=(0.0, 0.0, -g))
    ctx = erpp.Context(p, precision="fp64", weights=weights)
    fl = erpp.StokesFluid(p, precision="fp64")
    x0 = np.array([[1.1], [2.3], [3.7]])
    ps = erpp.ParticleState(cuda(x0), cuda(np.zeros((3, 1))), cuda(x0), cuda(np.zeros((3, 1))),
                            cuda(np.array([d / 2])), cuda(np.array([rho_ratio])))
    u = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
    S = ctx.new_grid()
    for k in range(120):
        ctx.step(u, ps, S=S, first_step=(k == 0))
        fl.step(u, S)
    ctx.check()
    return abs(-float(ps.v[2, 0]) / vt - 1.0)


def test_pic_settling_misses_the_terminal_velocity(erpp):
    ratios = GOLD["dp_over_sigmaR"]          # d_p / Dx with sigma_R = Dx
    pic = [_settle(erpp, r, "pic") for r in ratios]
    erpp_err = [_settle(erpp, r, "gaussian") for r in ratios]
    assert all(a > 2 * b for a, b in zip(pic, erpp_err)), (pic, erpp_err)
    assert all(a > b for a, b in zip(pic, pic[1:])), pic
    # the point-value gather with its own self removal stays near the ERPP run
    point = _settle(erpp, 0.5, "point")
    assert abs(point - erpp_err[0]) < 0.02 and point < 0.6 * pic[0], (point, erpp_err[0], pic[0])

"""GPU parity of the delayed source (ERPP_LAG) against the oracle
(oracle/lagged.py): the source of step n is D^(n-L) at x^(n-L), L =
round(eps_R / dt).

* several steps past L + 1 (no source, then source without removal, then
  both) with the field frozen: source, velocity and force per step within
  1e-5 (FP32, relative L2) and 1e-11 (FP64);
* ten steps of the closed loop through the GPU fluid stand-in: 1e-4 / 1e-11;
* the host-data step (erpp_step_host) carries the same history;
* coupled settling (Sec. 3.2.2) with the delay: the paper's claims;
* a changed particle count between first steps is refused.
"""

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


def _case():
    # dt = eps_R / 3 (L = 3) is large here (0.64): particles of radius 0.05
    # (tau_p = 55) keep the explicit Euler step far inside its stability range
    w = dataclasses.replace(
        I.CFG_SMALL.scaled("lag", (40, 36, 28), 700,
                           L=(2 * math.pi * 40 / 32, 2 * math.pi * 36 / 32,
                              2 * math.pi * 28 / 32)), radius=0.05)
    p = w.params(dt=w.eps_R / 3.0, gravity=(0.0, 0.007, -0.02))
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    return w, p, grid, st


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_lagged_steps_match_oracle(erpp, oracle_lib, precision):
    from oracle import lagged as LG
    w, p, grid, st = _case()
    assert LG.lag_steps(p) == 3
    ctx = erpp.Context(p, precision=precision, lag=True)
    ps = erpp.ParticleState.from_numpy(st)
    u = cuda(grid, _dtype(precision))
    S = ctx.new_grid()
    ref, h = st.copy(), LG.History()
    tol = 1e-5 if precision == "fp32" else 1e-11
    for n in range(9):
        ctx.step(u, ps, S=S, first_step=(n == 0))
        S_ref = LG.step(p, grid, ref, h, first_step=(n == 0))
        got = S.cpu().numpy()
        if n < 3:
            assert float(np.abs(got).max()) == 0.0, n
        else:
            assert rel(got, S_ref) < tol, n
        for name in ("v", "D"):
            assert rel(getattr(ps, name).cpu().numpy(), getattr(ref, name)) < tol, (n, name)
    ctx.check()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_lagged_coupled_loop_matches_oracle(erpp, oracle_lib, precision):
    from oracle import lagged as LG
    from oracle.stokes import stokes_step
    w, p, grid, st = _case()
    ctx = erpp.Context(p, precision=precision, lag=True)
    fl = erpp.StokesFluid(p, precision=precision)
    ps = erpp.ParticleState.from_numpy(st)
    u = cuda(grid, _dtype(precision))
    S = ctx.new_grid()
    ref, h, u_ref = st.copy(), LG.History(), grid.copy()
    for n in range(10):
        ctx.step(u, ps, S=S, first_step=(n == 0))
        fl.step(u, S)
        S_ref = LG.step(p, u_ref, ref, h, first_step=(n == 0))
        u_ref = stokes_step(u_ref, S_ref, p["nu"], p["dt"], w.L)
    ctx.check()
    tol = 1e-4 if precision == "fp32" else 1e-11
    assert rel(u.cpu().numpy(), u_ref) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol
    assert rel(ps.D.cpu().numpy(), ref.D) < tol


def test_lagged_host_step_keeps_the_history(erpp, oracle_lib):
    import torch
    w, p, grid, st = _case()
    dev = erpp.Context(p, precision="fp64", lag=True)
    host = erpp.Context(p, precision="fp64", lag=True)
    ps = erpp.ParticleState.from_numpy(st)
    ph = erpp.ParticleState.from_numpy(st).pinned()
    u = cuda(grid)
    uh = torch.as_tensor(grid).contiguous().pin_memory()
    S = dev.new_grid()
    Sh = torch.empty(tuple(S.shape), dtype=torch.float64).pin_memory()
    for n in range(6):
        dev.step(u, ps, S=S, first_step=(n == 0))
        host.step_host(uh, ph, Sh, first_step=(n == 0))
        host.step_host_wait()
    torch.cuda.synchronize()
    assert rel(Sh.numpy(), S.cpu().numpy()) < 1e-14
    assert rel(ph.D.numpy(), ps.D.cpu().numpy()) < 1e-14


def test_lagged_settling_claims(erpp):
    import torch

    def settle(dps, removal=True):
        L = 2 * math.pi
        N, nu, rho_ratio = 24, 0.1, 1000.0
        dx = L / N
        d = dps * dx
        tau = rho_ratio * d * d / (18 * nu)
        vt = 1e-3
        g = vt / tau / (1 - 1 / rho_ratio)
        p = dict(n=(N, N, N), L=(L, L, L), nu=nu, rho_f=1.0, eps_R=dx ** 2 / (2 * nu),
                 cutoff=3.0, dt=tau / 20, gravity=(0.0, 0.0, -g))
        ctx = erpp.Context(p, precision="fp64", self_removal=removal, lag=True)
        fl = erpp.StokesFluid(p, precision="fp64")
        x0 = np.array([[1.1], [2.3], [3.7]])
        ps = erpp.ParticleState(cuda(x0), cuda(np.zeros((3, 1))), cuda(x0),
                                cuda(np.zeros((3, 1))), cuda(np.array([d / 2])),
                                cuda(np.array([rho_ratio])))
        u = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
        S = ctx.new_grid()
        for k in range(120):
            ctx.step(u, ps, S=S, first_step=(k == 0))
            fl.step(u, S)
        ctx.check()
        return abs(-float(ps.v[2, 0]) / vt - 1.0)

    errs = [settle(r) for r in (0.5, 0.25, 0.125, 0.0625)]
    assert errs[0] < 0.10
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert settle(0.5, removal=False) > errs[0] + 0.01


def test_lagged_refuses_a_changed_particle_count(erpp):
    from paper_1405_6969_gb300 import ErppError
    w, p, grid, st = _case()
    ctx = erpp.Context(p, precision="fp64", lag=True)
    u = cuda(grid)
    S = ctx.new_grid()
    ctx.step(u, erpp.ParticleState.from_numpy(st), S=S, first_step=True)
    small = I.ParticleState(*(np.ascontiguousarray(a[..., :100]) for a in
                              (st.x, st.v, st.x_prev, st.D, st.radius, st.rho_p)))
    with pytest.raises(ErppError):
        ctx.step(u, erpp.ParticleState.from_numpy(small), S=S)
    # a first step with the new count starts a new history
    ctx.step(u, erpp.ParticleState.from_numpy(small), S=S, first_step=True)
    ctx.check()


def test_lagged_history_dropped_when_the_scratch_grows(erpp):
    """A call with more particles than the context has held reallocates its
    scratch, history included: the next step must be a first step."""
    from paper_1405_6969_gb300 import ErppError
    w, p, grid, st = _case()
    ctx = erpp.Context(p, precision="fp64", lag=True)
    u = cuda(grid)
    S = ctx.new_grid()
    ps = erpp.ParticleState.from_numpy(st)
    ctx.step(u, ps, S=S, first_step=True)
    ctx.step(u, ps, S=S)
    big = 2 * st.n + 2048
    rng = np.random.default_rng(5)
    xb = np.stack([rng.uniform(0, w.L[a], big) for a in range(3)])
    ctx.scatter_source(cuda(xb), cuda(np.zeros((3, big))), S=S)
    with pytest.raises(ErppError):
        ctx.step(u, ps, S=S)
    ctx.step(u, ps, S=S, first_step=True)
    ctx.check()

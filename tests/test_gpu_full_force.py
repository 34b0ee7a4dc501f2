"""GPU parity of the general force (ERPP_FULL_FORCE, Eq. force_particle)
against the oracle (oracle/full_force.py).

* several steps (the first without time derivatives or removal) in a random
  field, for particles of rho_p / rho_f = 2 and radius 0.05 (added mass,
  memory and Faxen terms all of visible size) and of rho_p / rho_f = 10 and
  radius 0.005 (drag-dominated): velocity, force and source per step within
  1e-11 (FP64) and, in FP32, within 1e-5 or the bound that the FP32 gather's
  rounding of u~ sets through the one-step differences of the force
  (`_fp32_bound`), whichever is larger;
* ten steps of the closed loop through the GPU fluid stand-in: 1e-4 / 1e-11;
* the Maxey-Riley steady slip in a uniformly accelerating fluid and the
  terminal velocity with buoyancy in coupled settling, on the GPU;
* a changed particle count without a first step is refused.
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


def _case(radius=0.05, rho_ratio=2.0):
    w = dataclasses.replace(
        I.CFG_SMALL.scaled("ff", (36, 32, 28), 500,
                           L=(2 * math.pi * 36 / 32, 2 * math.pi, 2 * math.pi * 28 / 32)),
        radius=radius, rho_ratio=rho_ratio)
    p = w.params(gravity=(0.0, -0.3, -1.0))
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    return w, p, grid, st


def _fp32_bound(p, st, ut, D):
    """Relative error of the force that the FP32 gather's rounding of u~
    causes through the terms that difference u~ over one step (Eq.
    force_particle: fluid acceleration m_f Du~/Dt, added mass (m_f/2) Du~/Dt
    and the one-step memory term, whose coefficient is
    c_B = 12 mu a^2 sqrt(pi / (nu dt))): u~ carries a rounding of about
    2^-24 |u~| at each step, the difference of two steps sqrt(2) times that,
    weighted by (3/2) m_f / dt + c_B against |D|; times 4 for the gather's
    sums, floored at the FP32 parity tolerance 1e-5."""
    a = st.radius
    m_f = (4.0 / 3.0) * math.pi * a ** 3 * p["rho_f"]
    mu = p["rho_f"] * p["nu"]
    c_B = 12.0 * mu * a ** 2 * math.sqrt(math.pi / (p["nu"] * p["dt"]))
    amp = np.linalg.norm(((1.5 * m_f / p["dt"] + c_B) * ut).ravel()) / np.linalg.norm(D.ravel())
    return max(1e-5, 4.0 * math.sqrt(2.0) * 2.0 ** -24 * amp)


@pytest.mark.parametrize("radius,rho_ratio", [(0.05, 2.0), (0.005, 10.0)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_force_steps_match_oracle(erpp, oracle_lib, precision, radius, rho_ratio):
    from oracle import full_force as FF
    w, p, grid, st = _case(radius, rho_ratio)
    ctx = erpp.Context(p, precision=precision, full_force=True)
    ps = erpp.ParticleState.from_numpy(st)
    u = cuda(grid, _dtype(precision))
    S = ctx.new_grid()
    ref, h = st.copy(), FF.History()
    for n in range(5):
        ctx.step(u, ps, S=S, first_step=(n == 0))
        S_ref = FF.step(p, grid, ref, h, first_step=(n == 0))
        if precision == "fp64":
            tol = 1e-11
        else:
            tol = 1e-5 if n == 0 else _fp32_bound(p, st, h.ut, ref.D)
            if rho_ratio == 10.0:
                # heavy, small particles: the drag dominates and the FP32
                # path meets the plain parity tolerance on every step
                assert tol == 1e-5, tol
        assert rel(S.cpu().numpy(), S_ref) < tol, n
        for name in ("v", "D"):
            assert rel(getattr(ps, name).cpu().numpy(), getattr(ref, name)) < tol, (n, name)
        # x^(n+1) = x^n + dt v^n: the velocity's tolerance carried over dt
        xtol = max(10 * p["dt"] * tol * np.abs(ref.v).max(), 1e-12)
        assert np.abs(ps.x.cpu().numpy() - ref.x).max() < xtol
    ctx.check()
    assert ctx.last_step_launches() >= 3


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_force_coupled_loop_matches_oracle(erpp, oracle_lib, precision):
    from oracle import full_force as FF
    from oracle.stokes import stokes_step
    w, p, grid, st = _case()
    ctx = erpp.Context(p, precision=precision, full_force=True)
    fl = erpp.StokesFluid(p, precision=precision)
    ps = erpp.ParticleState.from_numpy(st)
    u = cuda(grid, _dtype(precision))
    S = ctx.new_grid()
    ref, h, u_ref = st.copy(), FF.History(), grid.copy()
    for n in range(10):
        ctx.step(u, ps, S=S, first_step=(n == 0))
        fl.step(u, S)
        S_ref = FF.step(p, u_ref, ref, h, first_step=(n == 0))
        u_ref = stokes_step(u_ref, S_ref, p["nu"], p["dt"], w.L)
    ctx.check()
    tol = 1e-4 if precision == "fp32" else 1e-11
    assert rel(u.cpu().numpy(), u_ref) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol
    assert rel(ps.D.cpu().numpy(), ref.D) < tol


def _one(erpp, x0, a, rho_p):
    x = np.array(x0, dtype=np.float64)[:, None]
    return erpp.ParticleState(cuda(x), cuda(np.zeros((3, 1))), cuda(x), cuda(np.zeros((3, 1))),
                              cuda(np.array([a])), cuda(np.array([rho_p])))


def test_full_force_steady_slip_under_uniform_acceleration(erpp):
    """u = A t everywhere, no removal: the slip settles to (m_p - m_f) A /
    (6 pi mu a) (the added-mass, fluid-acceleration and drag balance)."""
    import torch
    p = dict(n=(20, 18, 16), L=(2.0, 1.8, 1.6), nu=0.05, rho_f=1.3,
             eps_R=(0.1 ** 2) / (2 * 0.05), cutoff=3.0, dt=2e-3)
    A = np.array([0.4, -0.2, 0.1])
    a, rho_ratio = 0.02, 2.0
    ctx = erpp.Context(p, precision="fp64", self_removal=False, full_force=True)
    ps = _one(erpp, (0.7, 0.9, 0.5), a, rho_ratio * p["rho_f"])
    u = torch.zeros((3, 16, 18, 20), dtype=torch.float64, device="cuda")
    S = ctx.new_grid()
    steps = 4000
    for k in range(steps):
        u.copy_(torch.as_tensor(A * k * p["dt"], device="cuda")[:, None, None, None]
                .expand(3, 16, 18, 20))
        ctx.step(u, ps, S=S, first_step=(k == 0))
    ctx.check()
    mu = p["rho_f"] * p["nu"]
    m_f = (4 / 3) * math.pi * a ** 3 * p["rho_f"]
    steady = (rho_ratio - 1) * m_f * A / (6 * math.pi * mu * a)
    slip = A * (steps - 1) * p["dt"] - ps.v[:, 0].cpu().numpy()
    np.testing.assert_allclose(slip + A * p["dt"], steady, rtol=1e-6)


def test_full_force_settling_with_buoyancy(erpp):
    import torch

    def settle(dps):
        L = 2 * math.pi
        N, nu, rho_ratio = 24, 0.1, 5.0
        dx = L / N
        d = dps * dx
        a = d / 2
        tau = rho_ratio * d * d / (18 * nu)
        g = 1e-3 / tau
        p = dict(n=(N, N, N), L=(L, L, L), nu=nu, rho_f=1.0, eps_R=dx ** 2 / (2 * nu),
                 cutoff=3.0, dt=tau / 20, gravity=(0.0, 0.0, -g))
        ctx = erpp.Context(p, precision="fp64", full_force=True)
        fl = erpp.StokesFluid(p, precision="fp64")
        ps = _one(erpp, (1.1, 2.3, 3.7), a, rho_ratio)
        u = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
        S = ctx.new_grid()
        for k in range(240):
            ctx.step(u, ps, S=S, first_step=(k == 0))
            fl.step(u, S)
        ctx.check()
        m_f = (4 / 3) * math.pi * a ** 3
        vt = (rho_ratio - 1) * m_f * g / (6 * math.pi * nu * a)
        return abs(-float(ps.v[2, 0]) / vt - 1.0)

    errs = [settle(r) for r in (0.5, 0.25, 0.125)]
    assert errs[0] < 0.10
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def test_full_force_refusals(erpp):
    from paper_1405_6969_gb300 import ErppError
    w, p, grid, st = _case()
    with pytest.raises(ErppError):
        erpp.Context(p, precision="fp64", full_force=True, lag=True)
    ctx = erpp.Context(p, precision="fp64", full_force=True)
    u = cuda(grid)
    S = ctx.new_grid()
    with pytest.raises(ErppError):      # the first step of a context must be a first step
        ctx.step(u, erpp.ParticleState.from_numpy(st), S=S)
    ctx.step(u, erpp.ParticleState.from_numpy(st), S=S, first_step=True)
    small = I.ParticleState(*(np.ascontiguousarray(a[..., :50]) for a in
                              (st.x, st.v, st.x_prev, st.D, st.radius, st.rho_p)))
    with pytest.raises(ErppError):
        ctx.step(u, erpp.ParticleState.from_numpy(small), S=S)
    ctx.check()

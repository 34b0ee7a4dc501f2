"""GPU parity of the fluid stand-in (erpp_fluid_*) and of the coupled loop.

* one exact Stokes step against the oracle's NumPy step (relative L2 1e-5
  in FP32, 1e-12 in FP64);
* ten steps of the closed two-way loop (coupling step, then the Stokes step
  with the new source) against the oracle loop: FP64 within 1e-11, FP32
  within 1e-4 (ten compounding steps of the 1e-5 single-step bound);
* the coupled settling of one heavy particle (Sec. 3.2.2) through the CUDA
  path: the paper's printed claims, as the oracle test checks them.
"""

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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


def _dtype(precision):
    import torch
    return torch.float32 if precision == "fp32" else torch.float64


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_stokes_step_matches_oracle(erpp, precision):
    from oracle.stokes import stokes_step
    n, L = (48, 40, 27), (2 * math.pi, 5.0, 4.0)
    p = dict(n=n, L=L, nu=0.05, rho_f=1.0, eps_R=0.01, cutoff=3.0, dt=0.02)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((3, n[2], n[1], n[0]))
    S = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = stokes_step(u, S, p["nu"], p["dt"], L)
    fl = erpp.StokesFluid(p, precision=precision)
    ut = cuda(u, _dtype(precision))
    fl.step(ut, cuda(S, _dtype(precision)))
    assert rel(ut.cpu().numpy(), ref) < (1e-5 if precision == "fp32" else 1e-12)
    # the result is divergence free: k . u_hat = 0 on every mode
    uh = np.fft.fftn(ut.cpu().numpy().astype(np.float64), axes=(1, 2, 3))
    kx = 2 * np.pi * np.fft.fftfreq(n[0], d=L[0] / n[0])
    ky = 2 * np.pi * np.fft.fftfreq(n[1], d=L[1] / n[1])
    kz = 2 * np.pi * np.fft.fftfreq(n[2], d=L[2] / n[2])
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    # Nyquist planes of even axes are their own mirror images: the real
    # transform keeps only the real part of k . u there, skip them
    mask = np.ones(K.shape, bool)
    for ax, m in ((2, n[0]), (1, n[1]), (0, n[2])):
        if m % 2 == 0:
            idx = [slice(None)] * 3
            idx[ax] = m // 2
            mask[tuple(idx)] = False
    scale = np.abs(uh).max() * K.max()
    assert np.abs(div[mask]).max() < (1e-5 if precision == "fp32" else 1e-12) * scale


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_loop_matches_oracle(erpp, oracle_lib, precision):
    from oracle.stokes import stokes_step
    w = I.CFG_SMALL
    p = w.params(gravity=(0.0, 0.0, -2.0))
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    ctx = erpp.Context(p, precision=precision)
    fl = erpp.StokesFluid(p, precision=precision)
    u = cuda(grid, _dtype(precision))
    ps = erpp.ParticleState.from_numpy(st)
    S = ctx.new_grid()
    ref, u_ref = st.copy(), grid.copy()
    for k in range(10):
        ctx.step(u, ps, S=S, first_step=(k == 0))
        fl.step(u, S)
        S_ref = oracle_lib.step(p, u_ref, ref, first_step=(k == 0))
        u_ref = stokes_step(u_ref, S_ref, p["nu"], p["dt"], w.L)
    ctx.check()
    tol = 1e-4 if precision == "fp32" else 1e-11
    assert rel(u.cpu().numpy(), u_ref) < tol
    assert rel(S.cpu().numpy(), S_ref) < tol
    assert rel(ps.v.cpu().numpy(), ref.v) < tol
    assert rel(ps.D.cpu().numpy(), ref.D) < tol


def _settle_gpu(erpp, dp_over_sigma, precision, removal=True, N=24, sig_over_dx=1.0):
    import torch
    L = GOLD["box_length"]
    nu, rho_ratio = 0.1, 1000.0
    dx = L / N
    sig = sig_over_dx * dx
    d = dp_over_sigma * sig
    tau = rho_ratio * d * d / (18 * nu)
    vt = 1e-3
    g = vt / tau / (1 - 1 / rho_ratio)
    dt = tau / 20
    p = dict(n=(N, N, N), L=(L, L, L), nu=nu, rho_f=1.0, eps_R=sig ** 2 / (2 * nu),
             cutoff=3.0, dt=dt, gravity=(0.0, 0.0, -g))
    ctx = erpp.Context(p, precision=precision, self_removal=removal)
    fl = erpp.StokesFluid(p, precision=precision)
    x0 = np.array([[1.1], [2.3], [3.7]])
    ps = erpp.ParticleState(cuda(x0), cuda(np.zeros((3, 1))), cuda(x0), cuda(np.zeros((3, 1))),
                            cuda(np.array([d / 2])), cuda(np.array([rho_ratio])))
    u = torch.zeros((3, N, N, N), dtype=_dtype(precision), device="cuda")
    S = ctx.new_grid()
    for k in range(120):
        ctx.step(u, ps, S=S, first_step=(k == 0))
        fl.step(u, S)
    ctx.check()
    return abs(-float(ps.v[2, 0]) / vt - 1.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_settling_claims_on_gpu(erpp, precision):
    errs = [_settle_gpu(erpp, r, precision) for r in GOLD["dp_over_sigmaR"]]
    assert errs[0] < GOLD["terminal_velocity_error_bound_at_dp_over_sigmaR_0.5"]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.01
    assert _settle_gpu(erpp, 0.5, precision, removal=False) > errs[0] + 0.01
    e48 = _settle_gpu(erpp, 0.5, precision, N=48, sig_over_dx=2.0)
    assert abs(e48 - errs[0]) < 2e-3

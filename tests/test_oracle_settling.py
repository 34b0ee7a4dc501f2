"""Coupled settling of one heavy particle (Sec. 3.2.2): the printed claims
of the paper, held against the oracle step closed by an exact Stokes fluid
step.  Values from ``tests/golden/settling_coupled.json``.

Set-up (the paper gives no further numbers): periodic box 2 pi, sigma_R =
dx on 24^3, nu = 0.1, rho_p/rho_f = 1000, v_t = 1e-3 (Re_p ~ 1e-3),
dt = tau_p / 20, six relaxation times from rest."""

import json
import math
import os

import numpy as np
import pytest

import erpp_inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "settling_coupled.json")))


def _settle(oracle_lib, dp_over_sigma, removal=True, N=24, sig_over_dx=1.0):
    from oracle.stokes import stokes_step
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
             cutoff=3.0, dt=dt, gravity=(0.0, 0.0, -g), self_removal=removal)
    x0 = np.array([[1.1], [2.3], [3.7]])
    st = I.ParticleState(x=x0.copy(), v=np.zeros((3, 1)), x_prev=x0.copy(),
                         D=np.zeros((3, 1)), radius=np.array([d / 2]),
                         rho_p=np.array([rho_ratio]))
    u = np.zeros((3, N, N, N))
    for n in range(120):
        S = oracle_lib.step(p, u, st, first_step=(n == 0))
        u = stokes_step(u, S, nu, dt, (L, L, L))
    return abs(-st.v[2, 0] / vt - 1.0)


def test_coupled_settling_terminal_velocity(oracle_lib):
    errs = [_settle(oracle_lib, r) for r in GOLD["dp_over_sigmaR"]]
    # below the printed 10 % at d_p / sigma_R = 0.5
    assert errs[0] < GOLD["terminal_velocity_error_bound_at_dp_over_sigmaR_0.5"]
    # decreasing with d_p / sigma_R
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.01
    # removing the self disturbance helps
    assert _settle(oracle_lib, 0.5, removal=False) > errs[0] + 0.01
    # grid independence at fixed sigma_R: 24^3 vs 48^3 (sigma_R = 2 dx)
    e48 = _settle(oracle_lib, 0.5, N=48, sig_over_dx=2.0)
    assert abs(e48 - errs[0]) < 2e-3

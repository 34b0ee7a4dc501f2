"""Pins of the validation references (Sec. 3) that the GPU validation tests
compare the CUDA path with.

Each reference is checked through a route other than its own formula: two
formulas of the paper against each other (Eq. ref_velo_f_fixed against the
time integral of the App. A.2 Green tensor; Eq. vorticity_solution against the
curl of the Green tensor), the textbook steady Stokeslet as t -> infinity,
incompressibility, the impulse theorem (Eq. impulse_def), and brute-force
iteration of the stand-in fluid step.
"""

import math

import numpy as np
import pytest

from oracle import validation as V
from oracle.stokes import stokes_step

NU, RHO = 0.7, 1.3
MU = NU * RHO


def test_axial_closed_form_equals_green_tensor_quadrature():
    """Eq. ref_velo_f_fixed is the time integral of G_xx(r e_x, s) over
    [0, t] (the Green tensor of Eq. green_tensor, unit force along x)."""
    for r in (0.05, 0.3, 1.0, 2.5):
        for t in (0.01, 0.2, 3.0):
            closed = V.fixed_force_axial_velocity(r, t, NU, MU)
            quad = V.fixed_force_velocity(np.array([r, 0.0, 0.0]), 0.0, t, [1.0, 0.0, 0.0],
                                          NU, RHO)
            assert quad[0] == pytest.approx(closed, rel=1e-9)
            assert abs(quad[1]) + abs(quad[2]) < 1e-12 * abs(closed)
            # the same along -x (the profile is even in r_x)
            quad_m = V.fixed_force_velocity(np.array([-r, 0.0, 0.0]), 0.0, t,
                                            [1.0, 0.0, 0.0], NU, RHO)
            assert quad_m[0] == pytest.approx(closed, rel=1e-9)


def test_steady_limits_are_the_stokeslet():
    """t -> infinity: the steady Stokeslet F/(8 pi mu)(I/r + r r^T/r^3),
    1/(4 pi mu r) on the force's axis, 1/(8 pi mu r) across it; vorticity
    F x r / (4 pi mu r^3)."""
    r = 0.8
    # approached like 1 - (4 / (3 sqrt(pi))) eta_t, eta_t = r / sqrt(4 nu t)
    for t in (1e5, 1e9):
        eta = r / math.sqrt(4 * NU * t)
        assert V.fixed_force_axial_velocity(r, t, NU, MU) == pytest.approx(
            (1.0 - 4.0 * eta / (3.0 * math.sqrt(math.pi))) / (4 * math.pi * MU * r), rel=1e-6)
    rv = np.array([0.3, -0.5, 0.4])
    F = np.array([0.2, 1.0, -0.6])
    rr = np.linalg.norm(rv)
    stokeslet = (F / rr + rv * (rv @ F) / rr ** 3) / (8 * math.pi * MU)
    # the Green tensor's time integral converges like t^(-1/2): integrate far out
    got = V.fixed_force_velocity(rv, 0.0, 1e8, F, NU, RHO)
    np.testing.assert_allclose(got, stokeslet, rtol=2e-4)
    zeta = V.fixed_force_vorticity(rv[:, None], 0.0, math.inf, F, NU, RHO)[:, 0]
    np.testing.assert_allclose(zeta, np.cross(F, rv) / (4 * math.pi * MU * rr ** 3),
                               rtol=1e-13)


def test_green_tensor_divergence_free_and_vorticity():
    """The Green tensor applied to a force is solenoidal, and its curl is the
    impulse vorticity of Eq. vorticity_solution (fourth-order central
    differences)."""
    s = 0.05
    F = np.array([0.4, -1.1, 0.7])
    h = 1e-3
    for x0 in (np.array([0.12, 0.05, -0.2]), np.array([-0.4, 0.3, 0.25])):
        def u(x):
            return V.green_tensor(x, s, NU, RHO) @ F

        def d(a, comp):
            e = np.zeros(3)
            e[a] = h
            return (-u(x0 + 2 * e)[comp] + 8 * u(x0 + e)[comp] - 8 * u(x0 - e)[comp]
                    + u(x0 - 2 * e)[comp]) / (12 * h)

        div = sum(d(a, a) for a in range(3))
        curl = np.array([d(1, 2) - d(2, 1), d(2, 0) - d(0, 2), d(0, 1) - d(1, 0)])
        zeta = V.impulse_vorticity(x0[:, None], s, F, NU, RHO)[:, 0]
        scale = np.abs(zeta).max()
        assert abs(div) < 1e-8 * scale
        np.testing.assert_allclose(curl, zeta, rtol=0, atol=1e-8 * scale)


def test_fixed_force_vorticity_closed_form_equals_quadrature():
    from scipy import integrate
    F = np.array([1.0, 0.3, -0.2])
    for rv in (np.array([0.1, 0.2, -0.05]), np.array([-0.9, 0.4, 1.2])):
        for s0, s1 in ((0.0, 0.05), (0.01, 0.3), (0.2, 4.0)):
            closed = V.fixed_force_vorticity(rv[:, None], s0, s1, F, NU, RHO)[:, 0]
            quad = np.array([integrate.quad(
                lambda s: V.impulse_vorticity(rv[:, None], s, F, NU, RHO)[c, 0],
                s0, s1, epsabs=0, epsrel=1e-12, limit=400)[0] for c in range(3)])
            np.testing.assert_allclose(closed, quad, rtol=1e-10,
                                       atol=1e-12 * np.abs(quad).max())


def test_vorticity_moment_gives_the_impulse():
    """Eq. impulse_def: (rho_f/2) int r x zeta = F0 (s1 - s0) for the vorticity
    of a constant force seen between the diffusion times s0 and s1 (Saffman's
    impulse), summed on a grid that resolves the smallest width
    sqrt(2 nu s0) of the closed-form vorticity."""
    L = (6.0, 6.0, 6.0)
    n = (96, 96, 96)
    F = np.array([1.0, -0.5, 0.25])
    s0, s1 = 0.05, 0.25
    xp = np.array([3.01, 2.97, 3.05])
    r = V.node_offsets(n, L, xp).reshape(3, -1)
    zeta = V.fixed_force_vorticity(r, s0, s1, F, 0.05, RHO)
    dV = np.prod(L) / np.prod(n)
    I = V.vorticity_moment(zeta, r, dV, RHO)
    np.testing.assert_allclose(I, F * (s1 - s0), rtol=1e-9)


def test_fixed_force_loop_equals_iterated_stokes_steps():
    rng = np.random.default_rng(3)
    n, L = (12, 10, 8), (2.0, 1.7, 1.5)
    S = rng.standard_normal((3, n[2], n[1], n[0]))
    u = np.zeros_like(S)
    for _ in range(7):
        u = stokes_step(u, S, NU, 0.013, L)
    got = V.fixed_force_loop(S, 7, NU, 0.013, L)
    np.testing.assert_allclose(got, u, rtol=0, atol=1e-13 * np.abs(u).max())
    np.testing.assert_allclose(V.impulse(got, L, RHO), RHO * 7 * 0.013 * np.prod(L)
                               / np.prod(n) * S.reshape(3, -1).sum(1), rtol=1e-12)


def test_spectral_curl_of_a_trigonometric_field():
    L = (2 * math.pi, 4 * math.pi, 2 * math.pi)
    n = (16, 24, 12)
    xs = [np.arange(n[a]) * L[a] / n[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    u = np.stack([np.sin(Y / 2) * np.cos(Z), np.cos(X) * np.sin(2 * Z), np.sin(3 * X + Y / 2)])
    # curl by hand
    cx = 0.5 * np.cos(3 * X + Y / 2) - 2 * np.cos(X) * np.cos(2 * Z)
    cy = -np.sin(Y / 2) * np.sin(Z) - 3 * np.cos(3 * X + Y / 2)
    cz = -np.sin(X) * np.sin(2 * Z) - 0.5 * np.cos(Y / 2) * np.cos(Z)
    np.testing.assert_allclose(V.spectral_curl(u, L), np.stack([cx, cy, cz]), atol=1e-12)


def test_imposed_motion_reduces_to_fixed_force():
    """A particle at rest with a constant force: Eq. ref_velo_disturbance is
    the fixed-force response; a particle carried at constant velocity V with
    the field evaluated in its frame at the same offset equals the quadrature
    of the Green tensor at the moving offset (the definition, two routes)."""
    F = np.array([0.3, 1.0, -0.4])
    x = np.array([0.4, -0.1, 0.2])
    got = V.imposed_motion_velocity(x, 0.3, lambda tau: np.zeros(3), lambda tau: F, NU, RHO)
    ref = V.fixed_force_velocity(x, 0.0, 0.3, F, NU, RHO)
    np.testing.assert_allclose(got, ref, rtol=1e-8)
    # linearity in the force history: a force switched on at t1 equals the
    # fixed-force response over the shorter time
    t1 = 0.1
    got = V.imposed_motion_velocity(x, 0.3, lambda tau: np.zeros(3),
                                    lambda tau: F if tau >= t1 else 0 * F, NU, RHO,
                                    breakpoints=(t1,))
    ref = V.fixed_force_velocity(x, 0.0, 0.3 - t1, F, NU, RHO)
    np.testing.assert_allclose(got, ref, rtol=1e-8)


def test_green_tensor_near_the_origin(oracle_lib):
    """Across the switch to the Taylor series at z = r / (sqrt(2) sigma) = 1e-3
    the tensor is continuous, and at r = 0 it is -1/dt times App. A.5's
    closed form at the same variance (the C oracle's self disturbance)."""
    s = 0.02
    sig = math.sqrt(2 * NU * s)
    rh = np.array([0.6, -0.48, 0.64])
    for z in (2e-3, 5e-3, 1e-2):
        r = z * math.sqrt(2) * sig
        direct = V.green_tensor(r * rh, s, NU, RHO)
        below = V.green_tensor(0.999e-3 * math.sqrt(2) * sig * rh, s, NU, RHO)
        # the series carries z^2; compare it extrapolated against the direct form
        assert np.abs(direct - below).max() < 2 * z * z * np.abs(direct).max()
    r_in = 0.9e-3 * math.sqrt(2) * sig
    r_out = 1.1e-3 * math.sqrt(2) * sig
    np.testing.assert_allclose(V.green_tensor(r_in * rh, s, NU, RHO),
                               V.green_tensor(r_out * rh, s, NU, RHO), rtol=0,
                               atol=1e-6 * abs(V.green_tensor(r_out * rh, s, NU, RHO)).max())
    D = np.array([0.3, -0.2, 0.9])
    p = dict(n=(16, 16, 16), L=(2 * math.pi,) * 3, nu=NU, rho_f=RHO, eps_R=0.0,
             cutoff=3.0, dt=s)
    # the oracle's self disturbance uses s2 = 2 nu (eps_R + dt) + sigma_R^2
    # (sigma_R^2 = 2 nu eps_R = 0 here): variance 2 nu s, the same as G(., s)
    v0 = oracle_lib.self_velocity(p, np.zeros((3, 1)), D[:, None])[:, 0]
    np.testing.assert_allclose(-s * V.green_tensor(np.zeros(3), s, NU, RHO) @ D, v0,
                               rtol=1e-12)

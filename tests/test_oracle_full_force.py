"""Pins of the general-force oracle step (oracle/full_force.py, Eq.
force_particle).

* The Laplacian of the matching gather equals second central differences of
  the C oracle's gather in the particle position (normalised and raw
  weights; particles whose windows do not change within the differences).
* The Laplacian of App. A.5's disturbance equals the finite-difference
  Laplacian of the C oracle's closed form in r, and 2 d/ds2 of it by central
  differences in the variance.
* Uniformly accelerating fluid, u = A t (no gradients, no self removal): the
  slip settles to the Maxey-Riley steady slip (m_p - m_f) A / (6 pi mu a) of
  the drag, added-mass and fluid-acceleration balance (the Basset memory and
  the Faxen terms vanish there).
* Coupled settling with buoyancy (rho_p / rho_f = 5, the added mass and the
  memory active in the transient): the terminal velocity (m_p - m_f) g /
  (6 pi mu a) within the paper's 10% at d_p / sigma_R = 0.5, decreasing
  with d_p / sigma_R.
"""

import math

import numpy as np

import erpp_inputs as I


def _p(**kw):
    d = dict(n=(20, 18, 16), L=(2.0, 1.8, 1.6), nu=0.05, rho_f=1.3,
             eps_R=(0.1 ** 2) / (2 * 0.05), cutoff=3.0, dt=1e-3)
    d.update(kw)
    return d


def test_gather_laplacian_finite_differences(oracle_lib):
    from oracle import full_force as FF
    rng = np.random.default_rng(0)
    for normalize in (True, False):
        p = _p(normalize=normalize)
        n = p["n"]
        u = rng.standard_normal((3, n[2], n[1], n[0]))
        x = np.stack([rng.uniform(0, p["L"][a], 30) for a in range(3)])
        h = 1e-4
        lo, hi = oracle_lib.windows(p, x)
        keep = np.ones(x.shape[1], bool)
        for a in range(3):
            for sgn in (1, -1):
                xs = x.copy()
                xs[a] += sgn * h
                l2, h2 = oracle_lib.windows(p, xs)
                keep &= (l2 == lo).all(0) & (h2 == hi).all(0)
        x = x[:, keep]
        assert x.shape[1] >= 15
        g0 = oracle_lib.gather(p, x, u)
        fd = np.zeros_like(g0)
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a] += h
            xm[a] -= h
            fd += (oracle_lib.gather(p, xp, u) - 2 * g0 + oracle_lib.gather(p, xm, u)) / (h * h)
        lap = FF.gather_laplacian(p, x, u)
        np.testing.assert_allclose(lap, fd, rtol=0, atol=2e-5 * np.abs(lap).max())


def test_self_laplacian_two_routes(oracle_lib):
    from oracle import full_force as FF
    p = _p()
    s2 = (2 * p["nu"]) * (p["eps_R"] + p["dt"]) + (2 * p["nu"]) * p["eps_R"]
    rng = np.random.default_rng(1)
    sig = math.sqrt(s2)
    radii = sig * np.array([0.0, 0.05, 0.3, 0.69, 0.72, 1.4, 3.0, 6.0])
    dirs = rng.standard_normal((3, len(radii)))
    dirs /= np.linalg.norm(dirs, axis=0)
    r = dirs * radii
    D = rng.standard_normal((3, len(radii)))
    lap = FF.self_laplacian(p, r, D)
    # central differences in the variance, through the C closed form
    hs = 1e-4 * s2
    ds2 = (oracle_lib.self_velocity(p, r, D, s2=s2 + hs)
           - oracle_lib.self_velocity(p, r, D, s2=s2 - hs)) / (2 * hs)
    # the closed form's prefactor carries dt/rho_f only through -dt/rho_f: fixed
    np.testing.assert_allclose(lap, 2 * ds2, rtol=1e-6, atol=1e-9 * np.abs(lap).max())
    # finite-difference Laplacian in r (away from r = 0)
    h = 1e-3 * sig
    far = radii > 0.1 * sig
    fd = -6 * oracle_lib.self_velocity(p, r, D)
    for a in range(3):
        e = np.zeros((3, 1))
        e[a] = h
        fd += oracle_lib.self_velocity(p, r + e, D) + oracle_lib.self_velocity(p, r - e, D)
    fd /= h * h
    np.testing.assert_allclose(lap[:, far], fd[:, far], rtol=0, atol=1e-5 * np.abs(lap).max())


def _uniform_state(a, rho_p, x0=(0.7, 0.9, 0.5)):
    x = np.array(x0, dtype=np.float64)[:, None]
    return I.ParticleState(x=x.copy(), v=np.zeros((3, 1)), x_prev=x.copy(), D=np.zeros((3, 1)),
                           radius=np.array([a]), rho_p=np.array([rho_p]))


def test_steady_slip_in_uniformly_accelerating_fluid(oracle_lib):
    from oracle import full_force as FF
    p = _p(self_removal=False, dt=2e-3)
    n = p["n"]
    A = np.array([0.4, -0.2, 0.1])
    a, rho_ratio = 0.02, 2.0
    st = _uniform_state(a, rho_ratio * p["rho_f"])
    h = FF.History()
    for k in range(4000):
        t = k * p["dt"]
        u = np.broadcast_to((A * t)[:, None, None, None], (3, n[2], n[1], n[0])).copy()
        FF.step(p, u, st, h, first_step=(k == 0))
    t = 3999 * p["dt"]
    slip = A * t - st.v[:, 0]
    mu = p["rho_f"] * p["nu"]
    m_f = (4 / 3) * math.pi * a ** 3 * p["rho_f"]
    m_p = rho_ratio * m_f
    # the slip of the step's own u~ (A t) against the velocity before the step
    # update converges to the steady balance; after the update v has moved on
    # by A dt
    steady = (m_p - m_f) * A / (6 * math.pi * mu * a)
    np.testing.assert_allclose(slip + A * p["dt"], steady, rtol=1e-6)


def test_settling_with_buoyancy(oracle_lib):
    from oracle import full_force as FF
    from oracle.stokes import stokes_step

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
        st = _uniform_state(a, rho_ratio, x0=(1.1, 2.3, 3.7))
        h = FF.History()
        u = np.zeros((3, N, N, N))
        for k in range(240):
            S = FF.step(p, u, st, h, first_step=(k == 0))
            u = stokes_step(u, S, nu, p["dt"], (L, L, L))
        mu = nu
        m_f = (4 / 3) * math.pi * a ** 3
        vt = (rho_ratio - 1) * m_f * g / (6 * math.pi * mu * a)
        return abs(-st.v[2, 0] / vt - 1.0)

    errs = [settle(r) for r in (0.5, 0.25, 0.125)]
    assert errs[0] < 0.10
    assert all(a > b for a, b in zip(errs, errs[1:])), errs

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
  the drag, added-mass and fluid-acceleration balance.  The fluid-side added
  mass and memory enter that balance with the opposite sign of the
  particle-side ones, so the steady slip holds only when the two sides carry
  the same coefficients.
* Particle released in a uniform stream (u = U, no gradients): the velocity
  relaxes geometrically to U with the time constant
  (m_p + m_f/2 + 6 pi mu a^2 I(dt)/dt) / (6 pi mu a), I(dt) the integral of
  the memory kernel (pi nu s)^(-1/2) over the last step (by quadrature): the
  particle's added mass and its one-step memory (Eq. force_particle, memory
  limited to the last step, Sec. 2.5).  As dt -> 0 the memory's share falls
  like sqrt(dt) and the time constant tends to the added-mass one,
  (m_p + m_f/2) / (6 pi mu a).
* The force returned to the fluid is the particle's hydrodynamic force of
  Eq. particle_motion: m_p (v' - v) / dt = D + (m_p - m_f) g, step by step,
  in a random field with gravity and the self removal on.
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


def _memory_integral(nu, dt):
    """int_0^dt (pi nu s)^(-1/2) ds by quadrature (algebraic-singularity weight)."""
    from scipy.integrate import quad
    val, err = quad(lambda s: (math.pi * nu) ** -0.5, 0.0, dt, weight="alg", wvar=(-0.5, 0.0))
    assert err < 1e-12 * abs(val)
    return val


def test_relaxation_time_of_added_mass_and_memory(oracle_lib):
    """A particle at rest in a uniform stream U: Eq. force_particle with the
    memory over the last step gives (m_p + m_f/2 + c dt)(v' - v)/dt =
    6 pi mu a (U - v) with c dt = 6 pi mu a^2 I(dt)/dt, so
    U - v_n = U (1 - dt/tau)^n exactly, tau = (m_p + m_f/2 + c dt)/(6 pi mu a).
    A factor 2 in the memory, or an added-mass coefficient of 1 instead of
    1/2, moves tau by tens of percent here."""
    from oracle import full_force as FF
    a, rho_ratio = 0.02, 2.0
    U = np.array([0.3, -0.1, 0.05])
    taus, expect, tau_am = [], [], None
    for dt in (4e-3, 1e-3, 2.5e-4):
        p = _p(self_removal=False, dt=dt)
        n = p["n"]
        mu = p["rho_f"] * p["nu"]
        m_f = (4 / 3) * math.pi * a ** 3 * p["rho_f"]
        m_p = rho_ratio * m_f
        u = np.broadcast_to(U[:, None, None, None], (3, n[2], n[1], n[0])).copy()
        st = _uniform_state(a, rho_ratio * p["rho_f"])
        h = FF.History()
        nsteps = 40
        for k in range(nsteps):
            FF.step(p, u, st, h, first_step=(k == 0))
        # U - v_n = U (1 - dt/tau)^n, per component
        ratio = (U - st.v[:, 0]) / U
        tau = dt / (1.0 - ratio ** (1.0 / nsteps))
        mem = 6 * math.pi * mu * a * a * _memory_integral(p["nu"], dt) / dt
        t_exp = (m_p + 0.5 * m_f + mem * dt) / (6 * math.pi * mu * a)
        # (tau is extracted through a 40th root: a few 1e-9 of rounding)
        np.testing.assert_allclose(tau, t_exp, rtol=1e-7)
        # the memory is a sizeable part of the inertia at these steps
        assert mem * dt > 0.1 * (m_p + 0.5 * m_f)
        taus.append(tau[0])
        expect.append(t_exp)
        tau_am = (m_p + 0.5 * m_f) / (6 * math.pi * mu * a)
    # the memory's excess over the added-mass time constant halves when dt
    # falls by 4: it vanishes like sqrt(dt)
    ex = [t - tau_am for t in taus]
    np.testing.assert_allclose(ex[1] / ex[0], 0.5, rtol=1e-5)
    np.testing.assert_allclose(ex[2] / ex[1], 0.5, rtol=1e-5)


def test_fluid_side_coefficients_match_particle_side(oracle_lib):
    """The steady slip in a uniformly accelerating stream is
    (m_p - m_f) A / (6 pi mu a) for any density ratio, including a neutrally
    buoyant particle (zero slip): the fluid-side added mass and memory cancel
    the particle-side ones only with equal coefficients."""
    from oracle import full_force as FF
    A = np.array([0.4, -0.2, 0.1])
    a = 0.02
    for rho_ratio in (1.0, 3.0):
        p = _p(self_removal=False, dt=1e-3)
        n = p["n"]
        st = _uniform_state(a, rho_ratio * p["rho_f"])
        h = FF.History()
        nsteps = 3000
        for k in range(nsteps):
            t = k * p["dt"]
            u = np.broadcast_to((A * t)[:, None, None, None], (3, n[2], n[1], n[0])).copy()
            FF.step(p, u, st, h, first_step=(k == 0))
        t = (nsteps - 1) * p["dt"]
        slip = A * t - st.v[:, 0] + A * p["dt"]
        mu = p["rho_f"] * p["nu"]
        m_f = (4 / 3) * math.pi * a ** 3 * p["rho_f"]
        steady = (rho_ratio - 1.0) * m_f * A / (6 * math.pi * mu * a)
        np.testing.assert_allclose(slip, steady, rtol=1e-6, atol=1e-12)


def test_returned_force_is_the_particle_force(oracle_lib):
    from oracle import full_force as FF
    p = _p(gravity=(0.0, -2.0, 0.5))
    n = p["n"]
    rng = np.random.default_rng(4)
    u = 0.3 * rng.standard_normal((3, n[2], n[1], n[0]))
    npart = 12
    x = np.stack([rng.uniform(0, p["L"][a], npart) for a in range(3)])
    st = I.ParticleState(x=x.copy(), v=0.1 * rng.standard_normal((3, npart)), x_prev=x.copy(),
                         D=np.zeros((3, npart)), radius=rng.uniform(0.01, 0.04, npart),
                         rho_p=rng.uniform(0.5, 4.0, npart) * p["rho_f"])
    h = FF.History()
    m_f = (4 / 3) * math.pi * st.radius ** 3 * p["rho_f"]
    m_p = (4 / 3) * math.pi * st.radius ** 3 * st.rho_p
    g = np.array(p["gravity"])[:, None]
    for k in range(4):
        v0 = st.v.copy()
        u = u + 0.05 * rng.standard_normal(u.shape)  # the field changes between steps
        FF.step(p, u, st, h, first_step=(k == 0))
        lhs = m_p * (st.v - v0) / p["dt"]
        rhs = st.D + (m_p - m_f) * g
        np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * np.abs(rhs).max())

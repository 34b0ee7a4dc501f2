"""Pins of the delayed-source oracle step (oracle/lagged.py).

* Source indexing: with the particles driven one way (no removal, a frozen
  field) the trajectories do not depend on the source, so the delayed source
  of step n must equal, bit for bit, the undelayed oracle's source of step
  n - L, and vanish for n < L.
* Removal indexing: the disturbance the step removes (read back from its own
  drag, D^n = 6 pi mu a (u_p - v_self - v^n)) must be the field that the
  previous step's source alone leaves at the particle after one exact Stokes
  step (App. A.5), within the 3% of the truncated kernel (2.3% here), and
  clearly not the one of the sources one step earlier or later (over 30% off).
* Coupled settling (Sec. 3.2.2) with the delay: the paper's claims hold.
"""

import math

import numpy as np

import erpp_inputs as I


def test_source_is_the_undelayed_source_L_steps_later(oracle_lib):
    from oracle import lagged as LG
    w = I.CFG_SMALL
    p = w.params(dt=w.eps_R / 3.0, self_removal=False)   # L = 3
    L = LG.lag_steps(p)
    assert L == 3
    grid, field = I.make_grid(w)
    st0 = I.make_particles(w, field)
    a, b = st0.copy(), st0.copy()
    h = LG.History()
    ref = []
    for n in range(L + 4):
        S_lag = LG.step(p, grid, a, h, first_step=(n == 0))
        ref.append(oracle_lib.step(p, grid, b, first_step=(n == 0)))
        assert np.array_equal(a.x, b.x) and np.array_equal(a.D, b.D)
        if n < L:
            assert not S_lag.any()
        else:
            assert np.array_equal(S_lag, ref[n - L])
    # a first step starts a new history
    S = LG.step(p, grid, a, h, first_step=True)
    assert not S.any() and len(h.x) == 1


def _settling_setup(dp_over_sigma, dt_over_tau, N=24):
    L = 2 * math.pi
    nu, rho_ratio = 0.1, 1000.0
    dx = L / N
    d = dp_over_sigma * dx
    tau = rho_ratio * d * d / (18 * nu)
    vt = 1e-3
    g = vt / tau / (1 - 1 / rho_ratio)
    dt = tau * dt_over_tau
    p = dict(n=(N, N, N), L=(L, L, L), nu=nu, rho_f=1.0, eps_R=dx ** 2 / (2 * nu),
             cutoff=3.0, dt=dt, gravity=(0.0, 0.0, -g))
    x0 = np.array([[1.1], [2.3], [3.7]])
    st = I.ParticleState(x=x0.copy(), v=np.zeros((3, 1)), x_prev=x0.copy(), D=np.zeros((3, 1)),
                         radius=np.array([d / 2]), rho_p=np.array([rho_ratio]))
    return p, st, vt


def test_removed_disturbance_is_the_previous_source(oracle_lib):
    from oracle import lagged as LG
    from oracle.stokes import stokes_step
    # early settling with large steps: the force changes by tens of per cent
    # from step to step, so neighbouring sources differ clearly
    p, st, _ = _settling_setup(0.5, 0.25)
    L = LG.lag_steps(p)
    n_check = L + 3
    N, Lb, nu, dt = p["n"][0], p["L"], p["nu"], p["dt"]
    u = np.zeros((3, N, N, N))
    h = LG.History()
    for n in range(n_check):
        S = LG.step(p, u, st, h, first_step=(n == 0))
        u = stokes_step(u, S, nu, dt, Lb)
    xn, vn = st.x.copy(), st.v.copy()
    up = oracle_lib.gather(p, xn, u)
    LG.step(p, u, st, h)
    k_drag = 6 * math.pi * p["rho_f"] * nu * st.radius[0]
    applied = up - vn - st.D / k_drag

    def alone(j):
        Sj = oracle_lib.scatter(p, h.x[j], h.D[j])
        return oracle_lib.gather(dict(p, shear_rate=0.0), xn, stokes_step(np.zeros_like(Sj), Sj,
                                                                        nu, dt, Lb))

    exp = alone(n_check - 1 - L)
    err = np.abs(applied - exp).max() / np.abs(exp).max()
    assert err < 3e-2
    for j in (n_check - L, n_check - 2 - L):
        other = np.abs(applied - alone(j)).max() / np.abs(exp).max()
        assert other > 3 * err, (j, other, err)


def test_settling_claims_with_the_delay(oracle_lib):
    from oracle import lagged as LG
    from oracle.stokes import stokes_step

    def settle(dps, removal=True):
        p, st, vt = _settling_setup(dps, 1 / 20)
        p["self_removal"] = removal
        N, Lb = p["n"][0], p["L"]
        u = np.zeros((3, N, N, N))
        h = LG.History()
        for n in range(120):
            S = LG.step(p, u, st, h, first_step=(n == 0))
            u = stokes_step(u, S, p["nu"], p["dt"], Lb)
        return abs(-st.v[2, 0] / vt - 1.0)

    errs = [settle(r) for r in (0.5, 0.25, 0.125, 0.0625)]
    assert errs[0] < 0.10
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert settle(0.5, removal=False) > errs[0] + 0.01

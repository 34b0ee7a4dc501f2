"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle through a route that does not retype its own
formula: exact rational arithmetic, Poisson summation of the Gaussian, a
second closed form printed in the paper (the unsteady Green tensor,
App. A.2), direct numerical quadrature, asymptotic limits, the exact
solution of the discrete Euler recursion, and finite differences.
"""

import math

import numpy as np
import pytest

import erpp_inputs as I


def _p(**kw):
    d = dict(n=(16, 16, 16), L=(2 * math.pi,) * 3, nu=0.01, rho_f=1.0,
             eps_R=(2 * math.pi / 16) ** 2 / 0.02, cutoff=3.0, dt=1e-3)
    d.update(kw)
    return d


# ---------------------------------------------------------------- windows

def test_windows_match_exact_rational_membership(oracle_lib):
    """The window is exactly the set of nodes with |x_j - x_p| <= r_c,
    decided here in exact rational arithmetic on the FP64 inputs."""
    from fractions import Fraction as Fr
    p = _p(n=(20, 12, 9), L=(3.0, 2.0, 1.5), nu=0.05, eps_R=0.03)
    rng = np.random.default_rng(5)
    x = rng.random((3, 400)) * np.array(p["L"])[:, None]
    lo, hi = oracle_lib.windows(p, x)
    sigma = math.sqrt((2.0 * p["nu"]) * p["eps_R"])
    rc = Fr(p["cutoff"] * sigma)
    for a in range(3):
        N, L = p["n"][a], Fr(p["L"][a])
        dx = L / N
        for i in range(x.shape[1]):
            xa = Fr(float(x[a, i]))
            j0 = math.floor((xa - rc) / dx) - 2
            j1 = math.ceil((xa + rc) / dx) + 2
            inside = [j for j in range(j0, j1 + 1) if abs(j * dx - xa) <= rc]
            assert (lo[a, i], hi[a, i]) == (inside[0], inside[-1])


def test_windows_on_nodes_are_symmetric(oracle_lib):
    """dx, 1/dx and r_c exact in binary: a particle on a node gets the
    2c+1 = 7 nodes j-3..j+3 (both end nodes at distance exactly r_c)."""
    p = _p(n=(32, 32, 32), L=(8.0, 8.0, 8.0), nu=0.5, eps_R=0.0625)
    j = np.array([0, 5, 31, 17])
    x = np.stack([j * 0.25, (j + 1) * 0.25 % 8.0, (j + 2) * 0.25 % 8.0])
    lo, hi = oracle_lib.windows(p, x)
    np.testing.assert_array_equal(hi - lo, 6)
    np.testing.assert_array_equal(lo[0], j - 3)


# ------------------------------------------------------ kernel (weights)

def _alias_sum(k, sigma, dxv, xp, sign, qmax=2):
    """sum_q exp(-sigma^2 |k + s Q|^2 / 2) exp(i s' (k + s Q) . x_p)."""
    tot = 0.0
    rng_q = range(-qmax, qmax + 1)
    for qx in rng_q:
        for qy in rng_q:
            for qz in rng_q:
                Q = 2 * np.pi * np.array([qx / dxv[0], qy / dxv[1], qz / dxv[2]])
                kk = k + Q
                tot = tot + np.exp(-0.5 * sigma ** 2 * np.sum(kk * kk, axis=-1)) * \
                    np.exp(sign * 1j * (kk @ xp))
    return tot


def test_scatter_fourier_coefficients_untruncated(oracle_lib):
    """Poisson summation: the DFT of the untruncated raw source of one
    particle is -(D/rho_f)/dV sum_q exp(-sigma^2|k+Q|^2/2) exp(-i(k+Q).x_p)
    (Gaussian transform of the heat kernel, App. A.1)."""
    n = (16, 12, 10)
    L = (2 * math.pi, 1.5 * math.pi, 1.3 * math.pi)
    sig = 0.9 * L[0] / n[0]
    p = _p(n=n, L=L, eps_R=sig ** 2 / 0.02)
    xp = np.array([[1.234], [0.71], [3.9]])
    D = np.array([[0.3], [-1.1], [0.7]])
    S = oracle_lib.scatter(dict(p, normalize=False, untruncated=True), xp, D)
    dxv = np.array(L) / np.array(n)
    dV = float(np.prod(dxv))
    Sh = np.fft.fftn(S, axes=(1, 2, 3))  # sum_j S_j exp(-i k.x_j)
    mz, my, mx = np.meshgrid(*(np.fft.fftfreq(n[a], 1.0 / n[a]) for a in (2, 1, 0)),
                             indexing="ij")
    k = np.stack([2 * np.pi * mx / L[0], 2 * np.pi * my / L[1],
                  2 * np.pi * mz / L[2]], axis=-1)
    expect_scalar = _alias_sum(k, sig, dxv, xp[:, 0], -1) / dV
    for c in range(3):
        expect = -D[c, 0] * expect_scalar
        err = np.max(np.abs(Sh[c] - expect)) / np.max(np.abs(expect))
        assert err < 1e-13


def test_gather_band_limited_field_untruncated(oracle_lib):
    """On u = sum_k Re(a_k e^{ik.x}) the untruncated raw gather returns
    sum_k Re(a_k sum_q e^{i(k-Q).x_p} e^{-sigma^2|k-Q|^2/2}) (Poisson)."""
    w = I.CFG_SMALL.scaled("t", (24, 24, 24), 40)
    grid, field = I.make_grid(w, kmax=3.0)
    p = w.params(normalize=False, untruncated=True)
    x = I.uniform_positions(40, w.L, 3)
    up = oracle_lib.gather(p, x, grid)
    dxv = np.array(w.L) / np.array(w.n)
    expect = np.zeros_like(x)
    for i in range(x.shape[1]):
        tot = np.zeros(3, dtype=complex)
        for kk, a in zip(field.k, field.a):
            # sum over aliases of mode k evaluated at x_p (sign +)
            s = _alias_sum(kk[None, :], w.sigma_R, dxv, x[:, i], +1, qmax=1)[0]
            tot += a * s
        expect[:, i] = tot.real
    assert np.max(np.abs(up - expect)) < 1e-12 * np.max(np.abs(expect))


def test_untruncated_axis_mass_poisson(oracle_lib):
    """sum_j dx g(x_j - x_p) over all images equals
    1 + 2 sum_m exp(-2 pi^2 m^2 sigma^2/dx^2) cos(2 pi m s) (Poisson): checked
    on the particle momentum -(1/rho_f) M_p D_p of raw weights."""
    p = _p(n=(16, 16, 16), normalize=False, untruncated=True)
    dx = 2 * math.pi / 16
    sig = math.sqrt(2 * p["nu"] * p["eps_R"])
    for s in (0.0, 0.25, 0.37, 0.5):
        xp = np.array([[s * dx + 3 * dx], [0.0], [0.0]])
        D = np.array([[-1.0], [0.0], [0.0]])
        S = oracle_lib.scatter(p, xp, D)
        _, Pp = oracle_lib.momentum(p, xp, D, S)
        axis = [1 + 2 * sum(math.exp(-2 * math.pi ** 2 * m * m * sig ** 2 / dx ** 2)
                            * math.cos(2 * math.pi * m * ss) for m in range(1, 4))
                for ss in (s, 0.0, 0.0)]
        assert abs(Pp[0] - np.prod(axis)) < 1e-14
        # the deficit is the Poisson term 2 exp(-2 pi^2) ~ 5.4e-9 at sigma = dx
        assert abs(Pp[0] - 1.0) > 1e-9 or s in (0.25,)


# ------------------------------------------------ conservation, transpose

@pytest.mark.parametrize("normalize", [True, False])
def test_momentum_conservation(oracle_lib, normalize):
    """Grid impulse of the source equals minus the particle forces (Sec. 3.1,
    I = F t): dV sum_j S_j = -(1/rho_f) sum_p M_p D_p."""
    w = I.CFG_SMALL
    p = w.params(normalize=normalize)
    st = I.make_particles(w, None, n_particles=300)
    S = oracle_lib.scatter(p, st.x, st.D)
    Pg, Pp = oracle_lib.momentum(p, st.x, st.D, S)
    np.testing.assert_allclose(Pg, Pp, rtol=1e-12, atol=1e-12 * np.abs(Pp).max())
    if normalize:
        np.testing.assert_allclose(Pp, -st.D.sum(axis=1), rtol=1e-13)


def test_gather_is_transpose_of_scatter(oracle_lib):
    """dV sum_j S_j . u_j = -(1/rho_f) sum_p D_p . (u_p - shear y_p e_x)."""
    w = dataclass_replace(I.CFG_CLUSTERED, n=(24, 20, 16))
    p = w.params()
    grid, _ = I.make_grid(w, kmax=4.0)
    st = I.make_particles(w, None, n_particles=200)
    S = oracle_lib.scatter(p, st.x, st.D)
    up = oracle_lib.gather(p, st.x, grid)
    up[0] -= w.shear_rate * st.x[1]
    dV = np.prod(np.array(w.L) / np.array(w.n))
    lhs = dV * np.sum(S * grid)
    rhs = -np.sum(st.D * up) / w.rho_f
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(st.D * up))


def dataclass_replace(w, **kw):
    import dataclasses
    return dataclasses.replace(w, **kw)


# ------------------------------------------------------------- self term

def _s2(p):
    return 2 * p["nu"] * (p["eps_R"] + p["dt"]) + 2 * p["nu"] * p["eps_R"]


def _green_tensor_velocity(r, D, s2, dt, rho_f):
    """-dt G_ik(r) D_k with the unsteady Green tensor of App. A.2
    (Eq. green_tensor) at variance s2."""
    from scipy.special import erf
    rr = np.linalg.norm(r)
    sig = math.sqrt(s2)
    g = (2 * math.pi * s2) ** -1.5 * math.exp(-rr * rr / (2 * s2))
    G = -erf(rr / (math.sqrt(2) * sig)) / (4 * math.pi * rr)
    A = (1 + s2 / rr ** 2) * g + G / rr ** 2
    B = (1 + 3 * s2 / rr ** 2) * g + 3 * G / rr ** 2
    Gik = (A * np.eye(3) - B * np.outer(r, r) / rr ** 2) / rho_f
    return -dt * Gik @ D


def _random_rD(n, scale, seed):
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    return dirs * scale, rng.standard_normal((3, n))


def test_self_velocity_equals_green_tensor(oracle_lib):
    """App. A.5's closed form equals -dt times the App. A.2 Green tensor at
    the same variance (two independent formulas of the paper)."""
    p = _p()
    s2 = _s2(p)
    radii = math.sqrt(s2) * np.array([0.5, 0.8, 1.0, 1.7, 2.5, 4.0, 7.0])
    r, D = _random_rD(len(radii), radii, 1)
    v = oracle_lib.self_velocity(p, r, D)
    for i in range(len(radii)):
        e = _green_tensor_velocity(r[:, i], D[:, i], s2, p["dt"], p["rho_f"])
        np.testing.assert_allclose(v[:, i], e, rtol=1e-12, atol=1e-13 * np.abs(e).max())


def test_self_velocity_direct_quadrature(oracle_lib):
    """Leray projection of the diffused point force by quadrature:
    v = -(dt/rho_f)[D g - grad(D.grad psi)], lap psi = g,
    psi'(r) = r^-2 int_0^r g s^2 ds (no error function involved)."""
    from scipy.integrate import quad
    p = _p()
    s2 = _s2(p)
    norm = (2 * math.pi * s2) ** -1.5
    gf = lambda s: norm * math.exp(-s * s / (2 * s2))  # noqa: E731
    radii = math.sqrt(s2) * np.array([0.05, 0.3, 0.9, 1.5, 3.0, 5.0])
    r, D = _random_rD(len(radii), radii, 2)
    v = oracle_lib.self_velocity(p, r, D)
    for i, rr in enumerate(radii):
        integral, _ = quad(lambda s: gf(s) * s * s, 0.0, rr, epsabs=0, epsrel=2e-14,
                           limit=200)
        dpsi = integral / rr ** 2
        d2psi = gf(rr) - 2 * dpsi / rr
        rh = r[:, i] / rr
        Dv = D[:, i]
        hess_D = (dpsi / rr) * Dv + (d2psi - dpsi / rr) * (Dv @ rh) * rh
        e = -(p["dt"] / p["rho_f"]) * (Dv * gf(rr) - hess_D)
        np.testing.assert_allclose(v[:, i], e, rtol=1e-11, atol=1e-12 * np.abs(e).max())


def test_self_velocity_limits(oracle_lib):
    """r -> 0: -(2/3)(dt/rho_f) g_s(0) D.  r >> sigma: the potential dipole
    -(dt/rho_f)(-D + 3 (D.rh) rh)/(4 pi r^3) behind the eps_R/r^3 law of
    Sec. 2.3."""
    p = _p()
    s2 = _s2(p)
    D = np.array([[0.3], [-0.2], [0.9]])
    v0 = oracle_lib.self_velocity(p, np.zeros((3, 1)), D)
    e0 = -(2.0 / 3.0) * (p["dt"] / p["rho_f"]) * (2 * math.pi * s2) ** -1.5 * D
    np.testing.assert_allclose(v0, e0, rtol=1e-15)
    vt = oracle_lib.self_velocity(p, np.array([[1e-9], [0.0], [0.0]]) * math.sqrt(s2), D)
    np.testing.assert_allclose(vt, e0, rtol=1e-12)
    for rr_over in (9.0, 12.0):
        rr = rr_over * math.sqrt(s2)
        rh = np.array([0.48, -0.6, 0.64])
        v = oracle_lib.self_velocity(p, (rr * rh)[:, None], D)[:, 0]
        e = -(p["dt"] / p["rho_f"]) * (-D[:, 0] + 3 * (D[:, 0] @ rh) * rh) / (4 * math.pi * rr ** 3)
        np.testing.assert_allclose(v, e, rtol=1e-12)


def test_self_velocity_high_precision(oracle_lib):
    """Against the App. A.5 closed form evaluated in 40-digit arithmetic,
    across the small-distance series branch and the direct branch."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    p = _p()
    s2 = _s2(p)
    etas = [1e-4, 1e-2, 0.2, 0.4999999, 0.5, 0.5000001, 0.8, 2.0, 4.0]
    rh = np.array([2.0, -1.0, 2.0]) / 3.0
    D = np.array([0.5, 1.5, -0.7])
    for eta in etas:
        rr = eta * math.sqrt(2 * s2)
        v = oracle_lib.self_velocity(p, (rr * rh)[:, None], D[:, None])[:, 0]
        E = mp.mpf(eta)
        f = mp.sqrt(mp.pi) / 2 * mp.erf(E) - E * mp.exp(-E * E)
        F = f / (2 * E ** 3)
        e = mp.exp(-E * E)
        pref = -(mp.mpf(p["dt"]) / p["rho_f"]) / (2 * mp.pi * mp.mpf(s2)) ** mp.mpf(1.5)
        Ddr = float(D @ rh)
        ref = [float(pref * ((e - F) * D[a] - Ddr * (e - 3 * F) * rh[a])) for a in range(3)]
        np.testing.assert_allclose(v, ref, rtol=2e-14, atol=1e-15 * max(map(abs, ref)))


def test_self_disturbance_end_to_end(oracle_lib):
    """One particle forces an exact Stokes step (forcing, diffusion,
    projection as in App. A.5); the kernel gather of the resulting field at
    x_p + r is the closed form at s2 = 2 nu (eps_R + dt) + sigma_R^2.  The
    truncated normalised kernel is not exactly Gaussian, hence 2e-2."""
    from oracle.stokes import stokes_step
    w = I.CFG_SMALL.scaled("t", (48, 48, 48), 1)
    p = w.params(dt=0.05)
    xp = np.array([[2.01], [3.3], [1.7]])
    D = np.array([[0.4], [-0.3], [0.8]])
    S = oracle_lib.scatter(p, xp, D)
    u = stokes_step(np.zeros_like(S), S, p["nu"], p["dt"], w.L)
    rs = np.array([[0.0, 0.03, -0.05, 0.1], [0.0, 0.02, 0.04, -0.1], [0.0, -0.01, 0.0, 0.05]])
    up = oracle_lib.gather(dict(p, shear_rate=0.0), xp + rs, u)
    vs = oracle_lib.self_velocity(p, rs, np.repeat(D, rs.shape[1], axis=1))
    err = np.max(np.abs(up - vs)) / np.max(np.abs(vs))
    assert err < 2e-2
    # without the gather's own sigma_R^2 the same field is far off
    s2_point = 2 * p["nu"] * (p["eps_R"] + p["dt"])
    wrong = np.stack([_green_tensor_velocity(rs[:, i], D[:, 0], s2_point, p["dt"], p["rho_f"])
                      for i in range(1, rs.shape[1])], axis=1)
    err_wrong = np.max(np.abs(up[:, 1:] - wrong)) / np.max(np.abs(vs))
    assert err_wrong > 10 * err


# ------------------------------------------------------- drag and Euler

def test_euler_settling_exact_discrete_solution(oracle_lib):
    """u = 0, no removal: Euler gives v^n = v_t (1 - (1 - dt/tau_p)^n) with
    tau_p = rho_p d_p^2/(18 mu) and v_t = tau_p (1 - rho_f/rho_p) g, the
    discrete analogue of Eq. uncoupled_solution; x^n is its running sum."""
    w = I.CFG_SMALL.scaled("t", (16, 16, 16), 3)
    p = w.params(gravity=(0.0, 0.0, -9.81), self_removal=False, dt=2e-3)
    st = I.make_particles(w, None, n_particles=3)
    st.v[:] = 0.0
    st.radius[:] = [1e-3, 2e-3, 5e-4]
    st.rho_p[:] = [1000.0, 2500.0, 800.0]
    x0 = st.x.copy()
    u = np.zeros((3, 16, 16, 16))
    mu = p["rho_f"] * p["nu"]
    tau = st.rho_p * (2 * st.radius) ** 2 / (18 * mu)
    vt = tau * (1 - p["rho_f"] / st.rho_p) * -9.81
    r = 1 - p["dt"] / tau
    zsum = np.zeros(3)
    for n in range(1, 41):
        v_before = st.v[2].copy()
        zsum += v_before * p["dt"]
        oracle_lib.step(p, u, st, first_step=(n == 1))
        np.testing.assert_allclose(st.v[2], vt * (1 - r ** n), rtol=1e-12)
        # the force handed to the fluid is the Stokes drag on the slip
        np.testing.assert_allclose(st.D[2], -6 * math.pi * mu * st.radius * v_before,
                                   rtol=1e-12, atol=1e-30)
    z = np.mod(x0[2] + zsum, w.L[2])
    np.testing.assert_allclose(st.x[2], z, rtol=1e-12)
    np.testing.assert_array_equal(st.x[:2], x0[:2])
    # small dt: the Euler solution approaches v_t (1 - exp(-t/tau_p))
    t = 40 * p["dt"]
    np.testing.assert_allclose(st.v[2], vt * (1 - np.exp(-t / tau)), rtol=0.1)


def test_advance_uses_min_image_displacement(oracle_lib):
    """The self term sees x^n - x^(n-1) through the periodic wrap."""
    w = I.CFG_SMALL.scaled("t", (16, 16, 16), 2)
    p = w.params()
    L = w.L[0]
    x = np.array([[1e-4, 3.0], [1.0, 1.0], [2.0, 2.0]])
    xprev = np.array([[L - 2e-4, 3.0 - 3e-4], [1.0, 1.0], [2.0, 2.0]])
    D = np.ones((3, 2))
    rad = np.full(2, 1e-3)
    rho = np.full(2, 1000.0)
    up = np.zeros((3, 2))
    outs = []
    for xi, xpi in ((x, xprev),):
        st = I.ParticleState(x=xi.copy(), v=np.zeros((3, 2)), x_prev=xpi.copy(),
                             D=D.copy(), radius=rad, rho_p=rho)
        oracle_lib.advance(p, up, st)
        outs.append(st.D.copy())
    # both particles moved by +3e-4 along x: identical self terms and forces
    np.testing.assert_allclose(outs[0][:, 0], outs[0][:, 1], rtol=1e-9)


# ------------------------------------------------------------ adjoints

def _membership_stable(oracle_lib, p, x, h):
    ok = np.ones(x.shape[1], dtype=bool)
    lo0, hi0 = oracle_lib.windows(p, x)
    for a in range(3):
        for sgn in (-1, 1):
            xs = x.copy()
            xs[a] += sgn * h
            lo, hi = oracle_lib.windows(p, xs)
            ok &= np.all(lo == lo0, axis=0) & np.all(hi == hi0, axis=0)
    return ok


@pytest.mark.parametrize("normalize", [True, False])
def test_scatter_adjoint_finite_differences(oracle_lib, normalize):
    """dL/dx and dL/dD of L = sum (S - T)^2 against central differences."""
    w = I.CFG_SMALL.scaled("t", (20, 18, 16), 6)
    p = w.params(normalize=normalize)
    rng = np.random.default_rng(3)
    x = I.uniform_positions(6, w.L, 11)
    D = rng.standard_normal((3, 6))
    T = 0.5 * oracle_lib.scatter(p, I.uniform_positions(6, w.L, 12), rng.standard_normal((3, 6)))

    def loss(xx, DD):
        S = oracle_lib.scatter(p, xx, DD)
        return np.sum((S - T) ** 2)

    S = oracle_lib.scatter(p, x, D)
    dD, dx = oracle_lib.scatter_backward(p, x, D, 2 * (S - T))
    h = 1e-6
    stable = _membership_stable(oracle_lib, p, x, h)
    assert stable.sum() >= 4
    for i in np.nonzero(stable)[0]:
        for a in range(3):
            xp_, xm_ = x.copy(), x.copy()
            xp_[a, i] += h
            xm_[a, i] -= h
            fd = (loss(xp_, D) - loss(xm_, D)) / (2 * h)
            assert abs(fd - dx[a, i]) < 1e-6 * max(1.0, abs(fd))
            Dp_, Dm_ = D.copy(), D.copy()
            Dp_[a, i] += h
            Dm_[a, i] -= h
            fd = (loss(x, Dp_) - loss(x, Dm_)) / (2 * h)
            assert abs(fd - dD[a, i]) < 1e-6 * max(1.0, abs(fd))


def test_scatter_adjoint_dot_product(oracle_lib):
    """<J dD, R> = <dD, J^T R>: the source is linear in D."""
    w = I.CFG_SMALL.scaled("t", (20, 18, 16), 50)
    p = w.params()
    rng = np.random.default_rng(4)
    x = I.uniform_positions(50, w.L, 1)
    dD = rng.standard_normal((3, 50))
    R = rng.standard_normal((3, 16, 18, 20))
    lhs = np.sum(oracle_lib.scatter(p, x, dD) * R)
    gD, _ = oracle_lib.scatter_backward(p, x, np.zeros((3, 50)), R)
    rhs = np.sum(dD * gD)
    assert abs(lhs - rhs) < 1e-13 * np.sum(np.abs(dD * gD))


def test_gather_adjoint_finite_differences(oracle_lib):
    w = dataclass_replace(I.CFG_CLUSTERED, n=(20, 18, 16), n_particles=5)
    p = w.params()
    grid, _ = I.make_grid(w, kmax=4.0)
    x = I.uniform_positions(5, w.L, 21)
    rng = np.random.default_rng(9)
    G = rng.standard_normal((3, 5))

    def loss(xx, uu):
        return np.sum(oracle_lib.gather(p, xx, uu) * G)

    du, dx = oracle_lib.gather_backward(p, x, grid, G)
    h = 1e-6
    stable = _membership_stable(oracle_lib, p, x, h)
    for i in np.nonzero(stable)[0]:
        for a in range(3):
            xp_, xm_ = x.copy(), x.copy()
            xp_[a, i] += h
            xm_[a, i] -= h
            fd = (loss(xp_, grid) - loss(xm_, grid)) / (2 * h)
            assert abs(fd - dx[a, i]) < 1e-6 * max(1.0, abs(fd))
    # du: the gather is linear in u, so <du, du_probe> = loss(u_probe)
    probe = rng.standard_normal(grid.shape)
    lin = np.sum(oracle_lib.gather(dict(p, shear_rate=0.0), x, probe) * G)
    assert abs(np.sum(du * probe) - lin) < 1e-12 * abs(lin) + 1e-14


def test_scatter_nodes_matches_full_scatter(oracle_lib):
    """The node-sampled source is the full source read at those nodes."""
    w = dataclass_replace(I.CFG_CLUSTERED, n=(20, 18, 16))
    p = w.params()
    st = I.make_particles(w, None, n_particles=500)
    S = oracle_lib.scatter(p, st.x, st.D)
    rng = np.random.default_rng(0)
    nodes = np.stack([rng.integers(0, n, 64) for n in w.n])
    sub = oracle_lib.scatter_nodes(p, st.x, st.D, nodes)
    np.testing.assert_allclose(sub, S[:, nodes[2], nodes[1], nodes[0]], rtol=1e-13,
                               atol=1e-13 * np.abs(S).max())

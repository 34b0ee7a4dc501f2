"""Reference solutions of the paper's validation cases (Sec. 3), FP64.

TEST INFRASTRUCTURE: only the test suite uses this module.  It holds the
closed forms and quadratures that the paper compares the ERPP algorithm with,
and the exact solution of the discrete loop (scatter once, then repeated
exact Stokes steps) that a fixed force drives on a periodic grid:

* ``heat_kernel``, ``potential_G``, ``green_tensor``: the unsteady Stokes
  fundamental solution of App. A.2 (Eq. fundamental_phys, Eq. G_solution,
  Eq. green_tensor), a point impulse applied at time 0, evaluated at time s;
* ``fixed_force_axial_velocity``: Eq. ref_velo_f_fixed, the velocity along a
  constant point force switched on at t = 0 (Sec. 3.1), on the force's axis;
* ``fixed_force_velocity``: the same response at any point, the time integral
  of the Green tensor (Sec. 3.1) between two times, by quadrature;
* ``imposed_motion_velocity``: Eq. ref_velo_disturbance, the disturbance of
  a particle moving on a prescribed path (Sec. 3.2.1), by quadrature;
* ``impulse_vorticity``, ``fixed_force_vorticity``: the vorticity of a point
  impulse (Eq. vorticity_solution with Eq. fundamental_phys) and its time
  integral for a constant force, in closed form (incomplete gamma function);
* ``vorticity_moment``: the impulse as the vorticity moment, Eq. impulse_def;
* ``spectral_curl``: the curl of a periodic grid field by FFT;
* ``fixed_force_loop``: the periodic-grid field after n coupling steps with a
  particle held fixed, as the sum of the n exact Stokes steps of the oracle's
  stand-in fluid (geometric series of the per-mode decay);
* ``impulse``: rho_f times the integral of u over the box (Sec. 3.1).
"""

from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.special import erf, gammainc

from .stokes import wavenumbers


def heat_kernel(r, s, nu):
    """Eq. fundamental_phys: (4 pi nu s)^(-3/2) exp(-r^2 / (4 nu s))."""
    r = np.asarray(r, dtype=np.float64)
    return (4.0 * math.pi * nu * s) ** -1.5 * np.exp(-r * r / (4.0 * nu * s))


def potential_G(r, s, nu):
    """Eq. G_solution: the solution of lap G = g, -erf(r / sqrt(4 nu s)) / (4 pi r)."""
    r = np.asarray(r, dtype=np.float64)
    return -erf(r / math.sqrt(4.0 * nu * s)) / (4.0 * math.pi * r)


def green_tensor(rvec, s, nu, rho_f):
    """Eq. green_tensor: G_ik(r, s) for r = x - xi, s = t - tau > 0.

    ``rvec`` is [3] or [3, m]; returns [3, 3] or [3, 3, m].

    The two coefficients cancel to leading order as r -> 0; below
    z = r / (sqrt(2) sigma) = 1e-3 (sigma^2 = 2 nu s) they are taken from their
    Taylor series in z, derived from those of exp and erf:
    rho_f a = C (4/3 - (8/5) z^2), rho_f b = -(4/5) C z^2, C = g(0) / 2, so
    that G_ik(0, s) = (2/3) g(0, s) delta_ik / rho_f."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r2 = np.sum(rvec * rvec, axis=0)
    r = np.sqrt(r2)
    sig2 = 2.0 * nu * s
    z2 = r2 / (2.0 * sig2)
    small = z2 < 1e-6
    r2s = np.where(small, 1.0, r2)
    g = heat_kernel(r, s, nu)
    G = potential_G(np.where(small, 1.0, r), s, nu)
    C = 0.5 * (2.0 * math.pi * sig2) ** -1.5
    a = np.where(small, C * (4.0 / 3.0 - 1.6 * z2),
                 (1.0 + sig2 / r2s) * g + G / r2s) / rho_f
    # b / r^2, the coefficient of r_i r_k
    b_r2 = np.where(small, -0.4 * C / sig2,
                    ((1.0 + 3.0 * sig2 / r2s) * g + 3.0 * G / r2s) / r2s) / rho_f
    eye = np.eye(3) if rvec.ndim == 1 else np.eye(3)[:, :, None]
    return a * eye - b_r2 * np.einsum("i...,k...->ik...", rvec, rvec)


def fixed_force_axial_velocity(r, t, nu, mu):
    """Eq. ref_velo_f_fixed: the velocity component along a constant point
    force of unit magnitude, applied from t = 0, at distance r on its axis."""
    r = np.asarray(r, dtype=np.float64)
    eta = r / math.sqrt(4.0 * nu * t)
    e = erf(eta)
    bracket = e / (2.0 * eta * eta) - e - np.exp(-eta * eta) / (math.sqrt(math.pi) * eta) + 1.0
    return bracket / (4.0 * math.pi * mu * r)


def fixed_force_velocity(rvec, s0, s1, F0, nu, rho_f):
    """int_{s0}^{s1} G(r, s) F0 ds (Sec. 3.1: the response to a constant force
    is the time convolution of the Green tensor with it) at one point r != 0."""
    F0 = np.asarray(F0, dtype=np.float64)
    # split [s0, s1] at the decades of s around the diffusion time r^2 / nu so
    # that each piece sees a smooth, well-scaled integrand
    r2 = float(np.sum(np.asarray(rvec, dtype=np.float64) ** 2))
    cuts = [s0]
    c = r2 / nu * 1e-3
    while c < s1:
        if c > s0:
            cuts.append(c)
        c *= 10.0
    cuts.append(s1)
    out = np.zeros(3)
    for i in range(3):
        f = lambda s, i=i: float(green_tensor(rvec, s, nu, rho_f)[i] @ F0)  # noqa: E731
        for a, b in zip(cuts[:-1], cuts[1:]):
            out[i] += integrate.quad(f, a, b, epsabs=0.0, epsrel=1e-12, limit=400)[0]
    return out


def imposed_motion_velocity(x, t, xp_of_tau, D_of_tau, nu, rho_f, breakpoints=(),
                            shift=0.0):
    """Eq. ref_velo_disturbance: u_i(x, t) = int_0^t G_ik(x - x_p(tau), t - tau)
    D_k(tau) dtau, where D is the force the particle exerts on the fluid and
    x_p(tau), D(tau) are callables returning [3] arrays; by quadrature.

    ``shift`` > 0 evaluates the Green tensor at t - tau + shift instead: the
    regularised field, each impulse seen with the extra diffusion time
    (shift = eps_R for a source spread to the width sigma_R)."""
    x = np.asarray(x, dtype=np.float64)

    def f(tau, i):
        s = t - tau + shift
        if s <= 0.0:
            return 0.0
        return float(green_tensor(x - xp_of_tau(tau), s, nu, rho_f)[i] @ D_of_tau(tau))

    out = np.zeros(3)
    pts = sorted(b for b in breakpoints if 0.0 < b < t)
    for i in range(3):
        out[i], _ = integrate.quad(f, 0.0, t, args=(i,), epsabs=0.0, epsrel=1e-10,
                                   limit=800, points=pts or None)
    return out


def fixed_force_loop(S, nsteps, nu, dt, L):
    """The field after ``nsteps`` steps u <- exp(-nu k^2 dt) P (u + dt S) from
    rest with the source S held fixed (the oracle's stand-in fluid step of
    App. A.5's splitting, repeated).

    Every mode off the Nyquist planes of even axes evolves on its own and
    sums to dt P S_hat sum_{j=1}^{n} exp(-j nu k^2 dt), a finite geometric
    series (n on the mean mode).  On the Nyquist planes the mode -k (mod N)
    carries a wavevector that is not the negative of k's, so the real part
    that each step keeps couples the two; those modes are iterated step by
    step, exactly as the repeated step treats them."""
    n = (S.shape[3], S.shape[2], S.shape[1])
    shape = S.shape[1:]
    KX, KY, KZ = wavenumbers(n, L)
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    K2s = np.where(K2 == 0.0, 1.0, K2)
    Sh = np.fft.fftn(S, axes=(1, 2, 3))

    def project(v, kx, ky, kz, k2):
        kdv = (kx * v[0] + ky * v[1] + kz * v[2]) / k2
        return np.stack([v[0] - kx * kdv, v[1] - ky * kdv, v[2] - kz * kdv])

    a = nu * K2 * dt
    with np.errstate(invalid="ignore", divide="ignore"):
        series = np.where(a > 0.0, np.exp(-a) * -np.expm1(-nsteps * a) / -np.expm1(-a),
                          float(nsteps))
    uh = dt * series[None] * project(Sh, KX, KY, KZ, K2s)

    nyq = np.zeros(shape, dtype=bool)
    for ax, m in ((2, n[0]), (1, n[1]), (0, n[2])):
        if m % 2 == 0:
            sl = [slice(None)] * 3
            sl[ax] = m // 2
            nyq[tuple(sl)] = True
    if nyq.any() and nsteps > 0:
        idx = np.nonzero(nyq)
        lin = np.ravel_multi_index(idx, shape)
        mir = tuple((-i) % m for i, m in zip(idx, shape))
        perm = np.searchsorted(lin, np.ravel_multi_index(mir, shape))
        kx, ky, kz, k2 = KX[idx], KY[idx], KZ[idx], K2s[idx]
        decay = np.exp(-a[idx])
        s = Sh[(slice(None),) + idx]
        v = np.zeros_like(s)
        for _ in range(nsteps):
            w = project(v + dt * s, kx, ky, kz, k2) * decay
            v = 0.5 * (w + np.conj(w[:, perm]))
        uh[(slice(None),) + idx] = v
    return np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))


def impulse(u, L, rho_f):
    """rho_f int u dV on the periodic grid (Sec. 3.1): rho_f dV sum_j u_j."""
    n = u.shape[1] * u.shape[2] * u.shape[3]
    dV = L[0] * L[1] * L[2] / n
    return rho_f * dV * np.asarray(u, dtype=np.float64).reshape(3, -1).sum(axis=1)


def impulse_vorticity(rvec, s, F0, nu, rho_f):
    """Vorticity at time s of the unit-time impulse F0 applied at r = 0:
    Eq. vorticity_solution, -(1/rho_f) F0 x grad g, with grad g = -r g / (2 nu s)
    from Eq. fundamental_phys.  ``rvec`` [3, m] -> [3, m]."""
    rvec = np.asarray(rvec, dtype=np.float64)
    F0 = np.asarray(F0, dtype=np.float64).reshape(3, 1)
    r = np.sqrt(np.sum(rvec * rvec, axis=0))
    g = heat_kernel(r, s, nu)
    return np.cross(F0, rvec, axis=0) * (g / (2.0 * nu * s * rho_f))


def fixed_force_vorticity(rvec, s0, s1, F0, nu, rho_f):
    """int_{s0}^{s1} of ``impulse_vorticity`` over s (0 <= s0 < s1 <= inf),
    in closed form: with q = r^2 / (4 nu s) the integrand becomes
    q^(1/2) e^(-q) / (2 nu pi^(3/2) r^3) dq, so the integral is
    (F0 x r) [P(3/2, q(s0)) - P(3/2, q(s1))] / (4 pi rho_f nu r^3),
    P the regularised lower incomplete gamma function."""
    rvec = np.asarray(rvec, dtype=np.float64)
    F0 = np.asarray(F0, dtype=np.float64).reshape(3, 1)
    r = np.sqrt(np.sum(rvec * rvec, axis=0))
    q0 = np.inf if s0 == 0.0 else r * r / (4.0 * nu * s0)
    q1 = 0.0 if math.isinf(s1) else r * r / (4.0 * nu * s1)
    fac = (gammainc(1.5, q0) - gammainc(1.5, q1)) / (4.0 * math.pi * rho_f * nu * r ** 3)
    return np.cross(F0, rvec, axis=0) * fac


def vorticity_moment(zeta, rvec, dV, rho_f):
    """Eq. impulse_def on grid samples: (rho_f / 2) sum_j r_j x zeta_j dV, with
    r_j the node positions relative to the origin of the moment; [3]."""
    zeta = np.asarray(zeta, dtype=np.float64).reshape(3, -1)
    rvec = np.asarray(rvec, dtype=np.float64).reshape(3, -1)
    return 0.5 * rho_f * dV * np.cross(rvec, zeta, axis=0).sum(axis=1)


def spectral_curl(u, L):
    """curl u of a periodic [3, nz, ny, nx] field, by FFT (i k x u_hat)."""
    n = (u.shape[3], u.shape[2], u.shape[1])
    KX, KY, KZ = wavenumbers(n, L)
    uh = np.fft.fftn(np.asarray(u, dtype=np.float64), axes=(1, 2, 3))
    w = np.stack([1j * (KY * uh[2] - KZ * uh[1]),
                  1j * (KZ * uh[0] - KX * uh[2]),
                  1j * (KX * uh[1] - KY * uh[0])])
    return np.real(np.fft.ifftn(w, axes=(1, 2, 3)))


def node_offsets(n, L, xp):
    """Minimum-image offsets x_j - x_p of every node, [3, nz, ny, nx]."""
    axes = [np.arange(n[a]) * (L[a] / n[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    r = np.stack([X - xp[0], Y - xp[1], Z - xp[2]])
    for a in range(3):
        r[a] = (r[a] + 0.5 * L[a]) % L[a] - 0.5 * L[a]
    return r

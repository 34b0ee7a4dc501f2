"""The general particle force of Eq. force_particle in the coupling step, FP64.

TEST INFRASTRUCTURE: only the test suite uses this module.  Eq. force_particle
(Sec. 2.5, after Maxey & Riley) adds to the Stokes drag the Faxen correction
(a^2/6) lap u~, the fluid-acceleration and added-mass terms and the Basset
memory, all on u~, the fluid velocity without the particle's own
disturbance.  The ERPP reading of Sec. 2.5 limits the memory integral to the
last step.  The discrete step written here (explicit Euler, the same order
as the Stokes-drag step; q = u~ + (a^2/6) L~ the Faxen-corrected velocity):

  u~ = u_p - v_self,   L~ = lap u_p - lap v_self                 (self removal)
  F  = 6 pi mu a (q - v)                                        (drag, Faxen)
     + m_f (u~ - u~_prev) / dt                                  (fluid acceleration)
     + (m_f/2) [(u~ + (a^2/10) L~) - (u~ + (a^2/10) L~)_prev] / dt
     + c_B (q - q_prev)                                         (Basset, fluid part)
  [(m_p + m_f/2) / dt + c_B] (v' - v) = F + (m_p - m_f) g
  D  = F - [(m_f/2) / dt + c_B] (v' - v)                        (the force the fluid returns)

with m_f = rho_f (4/3) pi a^3, c_B = 12 mu a^2 sqrt(pi / (nu dt)) and the
"_prev" values those of the previous step (equal to the current ones on a
first step: no time derivatives).  The Basset memory over the last step takes
the slip's rate constant over the step, int_0^dt (pi nu s)^(-1/2) ds =
2 sqrt(dt / (pi nu)); its particle part, like the added mass of the particle's
own acceleration, is taken at the step's velocity change v' - v (implicitly:
explicit, a memory coefficient c_B far above m_p / dt makes the step
unstable), its fluid part and the fluid-acceleration terms at the change of
u~ over the last step.  D u~/Dt is read along the particle path without its
convective part ((u~ - v) . grad u~, second order in the small slip of the
linear regime).

lap u_p is the Laplacian in the particle position of the matching kernel
gather (second derivatives of the per-axis weights, normalisation included);
lap v_self follows from App. A.5's closed form: the disturbance is the Leray
projection of a Gaussian of variance s2, and a Gaussian satisfies
d g / d s2 = (1/2) lap g, so lap v_self = 2 d v_self / d s2 at fixed dt/rho_f.
"""

from __future__ import annotations

import math

import numpy as np

from . import _f64, _params, gather, scatter


def _geom(p):
    n = [int(p.n[a]) for a in range(3)]
    L = [float(p.L[a]) for a in range(3)]
    sig2 = (2.0 * p.nu) * p.eps_R
    rc = p.cutoff * math.sqrt(sig2)
    inv_dx = [n[a] / L[a] for a in range(3)]
    dx = [L[a] / n[a] for a in range(3)]
    cp = [rc * inv_dx[a] for a in range(3)]
    return n, dx, inv_dx, cp, sig2


def axis_weights_d2(p, a, xa):
    """Window start, weights and their second derivatives in the particle
    coordinate, on axis a (normalised to unit discrete mass when
    p.normalize).  Returns (jlo, w, w2) with w, w2 arrays over the window."""
    n, dx, inv_dx, cp, sig2 = _geom(p)
    s = xa * inv_dx[a]
    jlo = int(math.ceil(s - cp[a]))
    jhi = int(math.floor(s + cp[a]))
    j = np.arange(jlo, jhi + 1, dtype=np.float64)
    d = (j - s) * dx[a]
    w = (1.0 / math.sqrt(2.0 * math.pi * sig2)) * np.exp(-(d * d) / (2.0 * sig2))
    # d w / d x_p = w d / sig2,  d2 w / d x_p2 = w (d^2 / sig2^2 - 1 / sig2)
    A = d / sig2
    B = d * d / (sig2 * sig2) - 1.0 / sig2
    if p.normalize:
        mass = dx[a] * w.sum()
        wn = w / mass
        m1 = dx[a] * (wn * A).sum()
        m2 = dx[a] * (wn * B).sum()
        return jlo, wn, wn * (B - 2.0 * A * m1 - m2 + 2.0 * m1 * m1)
    return jlo, w, w * B


def gather_laplacian(p, x, u):
    """lap_{x_p} of the matching kernel gather sum_j dV W_p(j) u_j, [3, m]."""
    p = _params(p)
    n, dx, _, _, _ = _geom(p)
    x = _f64(x)
    u = _f64(u, (3, n[2], n[1], n[0]))
    dV = dx[0] * dx[1] * dx[2]
    out = np.zeros_like(x)
    for i in range(x.shape[1]):
        lo, w, w2 = [], [], []
        for a in range(3):
            j0, wa, w2a = axis_weights_d2(p, a, x[a, i])
            lo.append(j0)
            w.append(wa)
            w2.append(w2a)
        iz = np.mod(lo[2] + np.arange(len(w[2])), n[2])
        iy = np.mod(lo[1] + np.arange(len(w[1])), n[1])
        ix = np.mod(lo[0] + np.arange(len(w[0])), n[0])
        block = u[:, iz][:, :, iy][:, :, :, ix]          # [3, kz, ky, kx]
        K = (np.einsum("z,y,x->zyx", w[2], w[1], w2[0]) +
             np.einsum("z,y,x->zyx", w[2], w2[1], w[0]) +
             np.einsum("z,y,x->zyx", w2[2], w[1], w[0]))
        out[:, i] = dV * np.einsum("czyx,zyx->c", block, K)
    return out


def _F_and_dF(eta):
    """F(eta) = f / (2 eta^3), f = (sqrt(pi)/2) erf(eta) - eta e^-eta^2, and
    dF/deta = e^-eta^2 / eta - 3 F / eta; Taylor series below eta = 1/2
    (F = sum_k (-1)^k eta^2k / (k! (2k+3)) term by term)."""
    from scipy.special import erf
    eta = np.asarray(eta, dtype=np.float64)
    F = np.empty_like(eta)
    dF = np.empty_like(eta)
    small = eta < 0.5
    e2 = eta[small] ** 2
    term = np.ones_like(e2)
    Fs = np.zeros_like(e2)
    dFs = np.zeros_like(e2)
    es = eta[small]
    for k in range(20):
        Fs += term / (2 * k + 3)
        if k >= 1:
            # d/deta of term / (2k+3) = 2k term / (eta (2k+3))
            dFs += 2 * k * term / (2 * k + 3)
        term = -term * e2 / (k + 1)
    F[small] = Fs
    dF[small] = np.where(es > 0, dFs / np.where(es > 0, es, 1.0), 0.0)
    el = eta[~small]
    f = 0.5 * math.sqrt(math.pi) * erf(el) - el * np.exp(-el * el)
    F[~small] = f / (2.0 * el ** 3)
    dF[~small] = np.exp(-el * el) / el - 3.0 * F[~small] / el
    return F, dF


def self_laplacian(p, r, D, s2=None):
    """lap of App. A.5's disturbance in r: 2 d v_self / d s2 (at the matching
    gather's variance unless s2 is given), [3, m].  With
    v = pref(s2) B(eta), pref ~ s2^(-3/2), eta = |r| / sqrt(2 s2):
    2 dv/ds2 = -(pref / s2) (3 B + eta dB/deta)."""
    p = _params(p)
    r, D = _f64(r), _f64(D)
    if s2 is None:
        s2 = (2.0 * p.nu) * (p.eps_R + p.dt) + (2.0 * p.nu) * p.eps_R
    pref = -(p.dt / p.rho_f) / (2.0 * math.pi * s2) ** 1.5
    rr = np.sqrt((r * r).sum(axis=0))
    eta = rr / math.sqrt(2.0 * s2)
    F, dF = _F_and_dF(eta)
    e = np.exp(-eta * eta)
    de = -2.0 * eta * e
    rh = np.where(rr > 0, r / np.where(rr > 0, rr, 1.0), 0.0)
    Ddr = (D * rh).sum(axis=0)
    B = (e - F) * D - Ddr * (e - 3.0 * F) * rh
    dB = (de - dF) * D - Ddr * (de - 3.0 * dF) * rh
    return -(pref / s2) * (3.0 * B + eta * dB)


class History:
    """u~ and L~ of the previous step, [3, n] each."""

    def __init__(self):
        self.ut = None
        self.Lt = None


def step(p, u, state, hist, first_step=False):
    """One coupling step with the general force, in place; returns S."""
    from . import self_velocity
    p = _params(p)
    if first_step:
        hist.ut = hist.Lt = None
    x, v = state.x, state.v
    up = gather(p, x, u)
    Lu = gather_laplacian(p, x, u)
    ut, Lt = up, Lu
    if p.self_removal and not first_step:
        r = x - state.x_prev
        for a in range(3):
            La = p.L[a]
            r[a] = np.where(r[a] > 0.5 * La, r[a] - La, np.where(r[a] < -0.5 * La, r[a] + La, r[a]))
        ut = up - self_velocity(p, r, state.D)
        Lt = Lu - self_laplacian(p, r, state.D)
    if hist.ut is None:
        hist.ut, hist.Lt = ut.copy(), Lt.copy()
    a_p = state.radius
    a2 = a_p * a_p
    mu = p.rho_f * p.nu
    dt = p.dt
    m_p = (4.0 / 3.0) * math.pi * a_p ** 3 * state.rho_p
    m_f = (4.0 / 3.0) * math.pi * a_p ** 3 * p.rho_f
    c_B = 12.0 * mu * a2 * math.sqrt(math.pi / (p.nu * dt))
    q = ut + (a2 / 6.0) * Lt
    q_prev = hist.ut + (a2 / 6.0) * hist.Lt
    F = (6.0 * math.pi * mu * a_p * (q - v)
         + m_f * (ut - hist.ut) / dt
         + 0.5 * m_f * ((ut + (a2 / 10.0) * Lt) - (hist.ut + (a2 / 10.0) * hist.Lt)) / dt
         + c_B * (q - q_prev))
    g = np.array([p.gravity[a] for a in range(3)])[:, None]
    dv = (F + (m_p - m_f) * g) / ((m_p + 0.5 * m_f) / dt + c_B)
    D = F - (0.5 * m_f / dt + c_B) * dv
    xn = x.copy()
    for a in range(3):
        La = p.L[a]
        xa = x[a] + dt * v[a]
        xa = np.where(xa < 0.0, xa + La, xa)
        x[a] = np.where(xa >= La, xa - La, xa)
    state.x_prev[...] = xn
    state.v[...] = v + dv
    state.D[...] = D
    hist.ut, hist.Lt = ut, Lt
    return scatter(p, state.x_prev, state.D)

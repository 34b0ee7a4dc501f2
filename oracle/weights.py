"""Other interpolation and projection weights on the same grid, FP64.

TEST INFRASTRUCTURE: only the test suite uses this module.  The paper
compares the ERPP coupling with the classical particle-in-cell (PIC) coupling
(Sec. 3.2.1 and 3.2.2: PIC panels of the imposed-motion and settling tests)
and discusses interpolating the fluid velocity at the particle point
(Sec. 2.5).  Written here as plain NumPy over particles:

* PIC (cloud in cell): the force of a particle goes to the 8 nodes of the
  grid cell that contains it with the trilinear weights
  w = prod_a (1 - |x_a - x_j,a| / dx_a), as a source density
  S_j = -(1/rho_f) sum_p D_p w_p(j) / dV, and the fluid velocity is
  interpolated at the particle with the same weights.  The self disturbance
  of PIC has no closed form: no removal (Sec. 3.2.2).
* point-value gather: the fluid velocity at the particle point by separable
  4-point Lagrange (cubic) interpolation over the nodes i0-1 .. i0+2 around
  it (i0 = floor(x / dx)).  Paired with the Gaussian source, the
  particle's own disturbance at its point is App. A.5's closed form at
  s2 = 2 nu (eps_R + dt), without the gather's sigma_R^2.

Positions in grid units are s = x * (N / L) (one rounding), i0 = floor(s),
f = s - i0; node indices wrap modulo N.  Grid fields are [3, nz, ny, nx].
"""

from __future__ import annotations

import numpy as np

from . import _params, _f64, advance, scatter, self_velocity


def _geom(p):
    n = [int(p.n[a]) for a in range(3)]
    L = [float(p.L[a]) for a in range(3)]
    inv_dx = [n[a] / L[a] for a in range(3)]
    dV = (L[0] / n[0]) * (L[1] / n[1]) * (L[2] / n[2])
    return n, L, inv_dx, dV


def cell(p, x):
    """(i0 [3, m] int64, f [3, m]) of every particle: the cell's lower node
    and the fractional offset in grid units."""
    p = _params(p)
    n, L, inv_dx, _ = _geom(p)
    x = _f64(x)
    for a in range(3):
        if not np.all((x[a] >= 0.0) & (x[a] < L[a])):
            raise ValueError("positions must lie in [0, L)")
    s = np.stack([x[a] * inv_dx[a] for a in range(3)])
    i0 = np.floor(s)
    return i0.astype(np.int64), s - i0


def trilinear_axis_weights(f):
    """Weights of the nodes i0, i0 + 1: (1 - f, f)."""
    return [1.0 - f, f]


def lagrange4_axis_weights(f):
    """Cubic Lagrange basis on the nodes i0-1, i0, i0+1, i0+2 (offsets
    -1, 0, 1, 2 from i0) evaluated at f in [0, 1)."""
    return [-(f * (f - 1.0) * (f - 2.0)) / 6.0,
            ((f + 1.0) * (f - 1.0) * (f - 2.0)) / 2.0,
            -((f + 1.0) * f * (f - 2.0)) / 2.0,
            ((f + 1.0) * f * (f - 1.0)) / 6.0]


def _stencil(p, x, kind):
    """Per particle: node indices [3][k] (wrapped) and weights [3][k]."""
    p = _params(p)
    n = [int(p.n[a]) for a in range(3)]
    i0, f = cell(p, x)
    if kind == "trilinear":
        offs, wf = (0, 1), trilinear_axis_weights
    else:
        offs, wf = (-1, 0, 1, 2), lagrange4_axis_weights
    idx = [[np.mod(i0[a] + o, n[a]) for o in offs] for a in range(3)]
    w = [wf(f[a]) for a in range(3)]
    return idx, w


def _nodes(p, x, kind):
    """Flattened node index and weight of every (particle, stencil node)."""
    p = _params(p)
    n = [int(p.n[a]) for a in range(3)]
    idx, w = _stencil(p, x, kind)
    k = len(idx[0])
    nodes, weights = [], []
    for kz in range(k):
        for ky in range(k):
            for kx in range(k):
                nodes.append((idx[2][kz] * n[1] + idx[1][ky]) * n[0] + idx[0][kx])
                weights.append(w[0][kx] * w[1][ky] * w[2][kz])
    return nodes, weights


def pic_scatter(p, x, D):
    """PIC source S_j = -(1/rho_f) sum_p D_p w_p(j) / dV, [3, nz, ny, nx]."""
    p = _params(p)
    n, _, _, dV = _geom(p)
    x, D = _f64(x), _f64(D)
    S = np.zeros((3, n[2] * n[1] * n[0]))
    nodes, weights = _nodes(p, x, "trilinear")
    for j, w in zip(nodes, weights):
        for c in range(3):
            np.add.at(S[c], j, -(D[c] / p.rho_f) * w / dV)
    return S.reshape(3, n[2], n[1], n[0])


def _gather(p, x, u, kind):
    p = _params(p)
    n, _, _, _ = _geom(p)
    x = _f64(x)
    u = _f64(u, (3, n[2], n[1], n[0])).reshape(3, -1)
    up = np.zeros_like(x)
    nodes, weights = _nodes(p, x, kind)
    for j, w in zip(nodes, weights):
        for c in range(3):
            up[c] += w * u[c][j]
    up[0] += p.shear_rate * x[1]
    return up


def pic_gather(p, x, u):
    """Trilinear interpolation of u at x, plus the mean shear along x."""
    return _gather(p, x, u, "trilinear")


def point_gather(p, x, u):
    """4-point Lagrange interpolation of u at x, plus the mean shear along x."""
    return _gather(p, x, u, "lagrange4")


def point_self_s2(p):
    """Variance of the self disturbance at the particle point: the forcing
    spread to sigma_R^2 = 2 nu eps_R and diffused one step (App. A.5)."""
    p = _params(p)
    return (2.0 * p.nu) * (p.eps_R + p.dt)


def step(p, u, state, kind, first_step=False):
    """One coupling step with other weights, in place; returns the source.

    kind "pic": trilinear gather, drag without self removal, Euler advance,
    PIC source of D^n at x^n.  kind "point": 4-point Lagrange gather, removal
    of the self disturbance at s2 = 2 nu (eps_R + dt) (none on the first
    step, as in the Gaussian step), drag, advance, Gaussian source."""
    from . import Params
    p = _params(p)
    q = Params.from_buffer_copy(p)
    q.self_removal = 0
    if kind == "pic":
        up = pic_gather(p, state.x, u)
    elif kind == "point":
        up = point_gather(p, state.x, u)
        if p.self_removal and not first_step:
            # minimum image, as the Gaussian step takes it
            r = state.x - state.x_prev
            for a in range(3):
                La = p.L[a]
                r[a] = np.where(r[a] > 0.5 * La, r[a] - La,
                                np.where(r[a] < -0.5 * La, r[a] + La, r[a]))
            up = up - self_velocity(p, r, state.D, s2=point_self_s2(p))
    else:
        raise ValueError(kind)
    advance(q, up, state, first_step=first_step)
    if kind == "pic":
        return pic_scatter(p, state.x_prev, state.D)
    return scatter(p, state.x_prev, state.D)

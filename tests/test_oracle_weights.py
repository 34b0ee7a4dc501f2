"""Pins of the oracle's PIC and point-value weights (oracle/weights.py).

Checked through routes other than their own formulas: polynomial
reproduction (linear for trilinear, cubic for 4-point Lagrange), fourth-order
convergence on a smooth field, brute force from the hat function of the
periodic node distance, momentum and the adjoint identity of the PIC source,
and an end-to-end exact Stokes step for the point-value self disturbance.
"""

import dataclasses
import math

import numpy as np
import pytest

import erpp_inputs as I


def _p(n=(12, 10, 14), L=(2.0, 1.7, 2.6), **kw):
    d = dict(n=n, L=L, nu=0.05, rho_f=1.3, eps_R=0.01, cutoff=3.0, dt=1e-3)
    d.update(kw)
    return d


def _interior(rng, m, p, lo_cells, hi_cells):
    """Positions whose cells keep lo_cells / hi_cells nodes below / above
    inside the box on every axis (no wrap-around)."""
    x = np.empty((3, m))
    for a in range(3):
        dx = p["L"][a] / p["n"][a]
        x[a] = rng.uniform(lo_cells * dx, p["L"][a] - (hi_cells + 1) * dx, m)
    return x


def _grid_coords(p):
    xs = [np.arange(p["n"][a]) * p["L"][a] / p["n"][a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def test_trilinear_reproduces_linear_fields(oracle_lib):
    from oracle import weights as W
    p = _p()
    rng = np.random.default_rng(0)
    x = _interior(rng, 200, p, 0, 1)
    X, Y, Z = _grid_coords(p)
    u = np.stack([0.3 + 1.1 * X - 0.4 * Y + 2.0 * Z, -0.7 * X + 0.2 * Z, 5.0 + 0.0 * X])
    up = W.pic_gather(p, x, u)
    np.testing.assert_allclose(up[0], 0.3 + 1.1 * x[0] - 0.4 * x[1] + 2.0 * x[2], atol=1e-13)
    np.testing.assert_allclose(up[1], -0.7 * x[0] + 0.2 * x[2], atol=1e-13)
    np.testing.assert_allclose(up[2], 5.0, atol=1e-13)


def test_lagrange4_reproduces_cubics_and_node_values(oracle_lib):
    from oracle import weights as W
    p = _p()
    rng = np.random.default_rng(1)
    x = _interior(rng, 200, p, 1, 2)
    X, Y, Z = _grid_coords(p)

    def f(X, Y, Z):
        return 0.5 - X ** 3 + 2 * X * Y * Z - 0.3 * Y ** 2 * Z + Z ** 3 * Y ** 3 / 7

    u = np.stack([f(X, Y, Z), f(Y, Z, X), f(Z, X, Y)])
    up = W.point_gather(p, x, u)
    np.testing.assert_allclose(up[0], f(x[0], x[1], x[2]), atol=1e-12)
    np.testing.assert_allclose(up[1], f(x[1], x[2], x[0]), atol=1e-12)
    np.testing.assert_allclose(up[2], f(x[2], x[0], x[1]), atol=1e-12)
    # on a node the interpolant is the node value (wrapping included)
    j = np.array([[0, 5, 11], [9, 0, 3], [13, 7, 0]])
    xn = np.stack([j[a] * p["L"][a] / p["n"][a] for a in range(3)])
    un = W.point_gather(p, xn, u)
    for c in range(3):
        np.testing.assert_allclose(un[c], u[c][j[2], j[1], j[0]], atol=1e-15)


def test_lagrange4_converges_at_fourth_order(oracle_lib):
    from oracle import weights as W
    rng = np.random.default_rng(2)
    errs = []
    for N in (16, 32, 64):
        p = _p(n=(N, N, N), L=(2 * math.pi,) * 3)
        X, Y, Z = _grid_coords(p)
        u = np.stack([np.sin(X + 2 * Y) * np.cos(Z), np.cos(X - Z), np.sin(Y) * np.sin(Z)])
        x = rng.uniform(0, 2 * math.pi, (3, 300))
        up = W.point_gather(p, x, u)
        ex = np.stack([np.sin(x[0] + 2 * x[1]) * np.cos(x[2]), np.cos(x[0] - x[2]),
                       np.sin(x[1]) * np.sin(x[2])])
        errs.append(np.abs(up - ex).max())
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20, errs


def test_pic_scatter_brute_force_hat_function(oracle_lib):
    """S_j = -(1/rho_f) sum_p D_p prod_a max(0, 1 - |d_a| / dx_a) / dV with d_a
    the periodic (minimum image) node distance: every node, every particle."""
    from oracle import weights as W
    p = _p(n=(6, 5, 7))
    rng = np.random.default_rng(3)
    m = 9
    x = np.stack([rng.uniform(0, p["L"][a], m) for a in range(3)])
    x[:, 0] = [0.0, 0.0, 0.0]                       # on the corner node
    x[0, 1] = p["L"][0] * (1 - 1e-16)               # next to the upper face
    D = rng.standard_normal((3, m))
    S = W.pic_scatter(p, x, D)
    n, L = p["n"], p["L"]
    dV = np.prod([L[a] / n[a] for a in range(3)])
    ref = np.zeros_like(S)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                node = (i, j, k)
                for q in range(m):
                    w = 1.0
                    for a in range(3):
                        dx = L[a] / n[a]
                        d = x[a, q] - node[a] * dx
                        d -= L[a] * round(d / L[a])
                        w *= max(0.0, 1.0 - abs(d) / dx)
                    ref[:, k, j, i] += -(D[:, q] / p["rho_f"]) * w / dV
    np.testing.assert_allclose(S, ref, atol=1e-12 * np.abs(ref).max())


def test_pic_momentum_and_adjoint(oracle_lib):
    from oracle import weights as W
    p = _p()
    rng = np.random.default_rng(4)
    x = np.stack([rng.uniform(0, p["L"][a], 50) for a in range(3)])
    D = rng.standard_normal((3, 50))
    S = W.pic_scatter(p, x, D)
    dV = np.prod([p["L"][a] / p["n"][a] for a in range(3)])
    np.testing.assert_allclose(S.reshape(3, -1).sum(1) * dV, -D.sum(1) / p["rho_f"], rtol=1e-13)
    u = rng.standard_normal(S.shape)
    lhs = float((S * u).sum() * dV)
    rhs = float(-(D * W.pic_gather(dict(p, shear_rate=0.0), x, u)).sum() / p["rho_f"])
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_point_gather_sees_the_self_disturbance_without_sigma(oracle_lib):
    """One particle forces one exact Stokes step; the point-value gather at
    x_p + r is App. A.5's closed form at s2 = 2 nu (eps_R + dt) (interpolation
    error aside, sigma_R = 3 dx), not at the matching-gather variance with
    sigma_R^2 added."""
    from oracle import weights as W
    from oracle.stokes import stokes_step
    # sigma_R = 3 dx: the cubic interpolant resolves the disturbance
    w = dataclasses.replace(I.CFG_SMALL.scaled("t", (64, 64, 64), 1), sigma_over_dx=3.0)
    p = w.params(dt=0.05)
    xp = np.array([[2.01], [3.3], [1.7]])
    D = np.array([[0.4], [-0.3], [0.8]])
    S = oracle_lib.scatter(p, xp, D)
    u = stokes_step(np.zeros_like(S), S, p["nu"], p["dt"], w.L)
    rs = np.array([[0.0, 0.03, -0.05, 0.1], [0.0, 0.02, 0.04, -0.1], [0.0, -0.01, 0.0, 0.05]])
    up = W.point_gather(dict(p, shear_rate=0.0), xp + rs, u)
    Dn = np.repeat(D, rs.shape[1], axis=1)
    vs = oracle_lib.self_velocity(p, rs, Dn, s2=W.point_self_s2(p))
    err = np.max(np.abs(up - vs)) / np.max(np.abs(vs))
    assert err < 2e-2
    wrong = oracle_lib.self_velocity(p, rs, Dn)
    assert np.max(np.abs(up - wrong)) / np.max(np.abs(vs)) > 10 * err

"""GPU parity of the hand-written adjoints of the source and of the gather.

The CUDA entry points erpp_scatter_backward / erpp_gather_backward (through
the autograd Functions of the binding) against the FP64 oracle's adjoints,
relative L2 within 1e-5 (FP32 context) or 1e-12 (FP64 context); the
128^3 / 100k-particle loss L = sum (S - T)^2 additionally against central
differences of the FP64 oracle.  Inputs come from ``erpp_inputs``, expected
values from ``oracle`` only.
"""

import dataclasses
import math

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def erpp(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_6969_gb300 as pkg
    return pkg


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


def grid_t(g, precision):
    import torch
    return cuda(g, torch.float32 if precision == "fp32" else torch.float64)


CASES = [
    ("cube32", dataclasses.replace(I.CFG_SMALL), 800),
    ("ragged_72x40x20_sigma1.5", dataclasses.replace(I.CFG_CLUSTERED, n=(72, 40, 20),
                                                     n_particles=1500, cluster_std=0.3), 1500),
    ("aniso_96x33x17", dataclasses.replace(I.CFG_SMALL, n=(96, 33, 17),
                                           L=(2 * math.pi, 2.0, 1.0)), 1200),
]


def _inputs(w, n):
    grid, _ = I.make_grid(w)
    x = I.uniform_positions(n, w.L, 5) if w.cloud == "uniform" else \
        I.clustered_positions(n, w.L, 10, 0.3, 5)
    rng = np.random.default_rng(6)
    D = rng.standard_normal((3, n))
    return grid, x, D, rng


@pytest.mark.parametrize("normalize", [True, False])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,w,n", CASES, ids=[c[0] for c in CASES])
def test_scatter_backward(erpp, oracle_lib, precision, normalize, name, w, n):
    p = w.params(normalize=normalize)
    _, x, D, rng = _inputs(w, n)
    R = rng.standard_normal((3,) + tuple(w.n[::-1]))
    ctx = erpp.Context(p, precision=precision, normalize=normalize)
    dD, dx = ctx.scatter_backward(cuda(x), cuda(D), grid_t(R, precision))
    ctx.check()
    rdD, rdx = oracle_lib.scatter_backward(p, x, D, R)
    assert rel(dD.cpu().numpy(), rdD) < TOL[precision]
    assert rel(dx.cpu().numpy(), rdx) < TOL[precision]


@pytest.mark.parametrize("normalize", [True, False])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,w,n", CASES, ids=[c[0] for c in CASES])
def test_gather_backward(erpp, oracle_lib, precision, normalize, name, w, n):
    p = w.params(normalize=normalize)
    grid, x, _, rng = _inputs(w, n)
    G = rng.standard_normal((3, n))
    ctx = erpp.Context(p, precision=precision, normalize=normalize)
    du, dx = ctx.gather_backward(cuda(x), grid_t(grid, precision), cuda(G))
    ctx.check()
    rdu, rdx = oracle_lib.gather_backward(p, x, grid, G)
    assert rel(du.cpu().numpy(), rdu) < TOL[precision]
    assert rel(dx.cpu().numpy(), rdx) < TOL[precision]


def test_backward_empty_and_optional_outputs(erpp, oracle_lib):
    import torch
    w = I.CFG_SMALL
    p = w.params()
    ctx = erpp.Context(p, precision="fp32")
    x0 = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    dD, dx = ctx.scatter_backward(x0, x0, ctx.new_grid().zero_())
    assert dD.shape == (3, 0) and dx.shape == (3, 0)
    du, _ = ctx.gather_backward(x0, ctx.new_grid().zero_(), x0, need_dx=False)
    assert float(du.abs().max()) == 0.0
    # dD not requested: dx alone still matches
    grid, x, D, rng = _inputs(w, 300)
    R = rng.standard_normal((3,) + tuple(w.n[::-1]))
    none, dx = ctx.scatter_backward(cuda(x), cuda(D), grid_t(R, "fp32"), need_dD=False)
    ctx.check()
    assert none is None
    assert rel(dx.cpu().numpy(), oracle_lib.scatter_backward(p, x, D, R)[1]) < 1e-5


def test_interpolate_autograd(erpp, oracle_lib):
    """d/d(u, x) of sum_p G_p . u_p through the Interpolate Function."""
    import torch
    w = dataclasses.replace(I.CFG_CLUSTERED, n=(48, 40, 36), shear_rate=0.7)
    p = w.params()
    grid, x, _, rng = _inputs(w, 2000)
    G = rng.standard_normal((3, 2000))
    ctx = erpp.Context(p, precision="fp32")
    u_t = grid_t(grid, "fp32").requires_grad_()
    x_t = cuda(x).requires_grad_()
    up = erpp.Interpolate.apply(ctx, u_t, x_t)
    (up * cuda(G)).sum().backward()
    ctx.check()
    rdu, rdx = oracle_lib.gather_backward(p, x, grid, G)
    assert rel(u_t.grad.cpu().numpy(), rdu) < 1e-5
    assert rel(x_t.grad.cpu().numpy(), rdx) < 1e-5


def _adjoint_workload():
    """128^3, 100k uniform particles, sigma_R = 1.5 dx; D ~ N(0, 1) (seed 1);
    target T = 0.5 S(x', D') of an independent cloud (seed 2)."""
    w = I.CFG_ADJOINT
    n = w.n_particles
    x = I.uniform_positions(n, w.L, 0)
    D = np.random.default_rng(1).standard_normal((3, n))
    x2 = I.uniform_positions(n, w.L, 2)
    D2 = np.random.default_rng(2).standard_normal((3, n))
    return w, x, D, x2, D2


def test_config_adjoint_128cube_autograd(erpp, oracle_lib):
    """L = sum (S - T)^2 at 128^3 / 100k: gradients through ScatterSource in
    FP32 against the FP64 oracle gradient, and against oracle central
    differences (h = 1e-4) for sampled particles."""
    import torch
    w, x, D, x2, D2 = _adjoint_workload()
    p = w.params()
    T = 0.5 * oracle_lib.scatter(p, x2, D2)
    S_ref = oracle_lib.scatter(p, x, D)
    rdD, rdx = oracle_lib.scatter_backward(p, x, D, 2.0 * (S_ref - T))

    ctx = erpp.Context(p, precision="fp32")
    x_t = cuda(x).requires_grad_()
    D_t = cuda(D).requires_grad_()
    S = erpp.ScatterSource.apply(ctx, x_t, D_t)
    loss = ((S.double() - cuda(T)) ** 2).sum()
    loss.backward()
    ctx.check()
    gx = x_t.grad.cpu().numpy()
    gD = D_t.grad.cpu().numpy()
    assert rel(gD, rdD) < 1e-5
    assert rel(gx, rdx) < 1e-5
    L_ref = float(np.sum((S_ref - T) ** 2))
    assert abs(float(loss.detach()) - L_ref) < 1e-5 * L_ref

    # central differences of the FP64 oracle loss, evaluated locally: moving
    # particle i changes S only on its stencil box
    h = 1e-4
    rng = np.random.default_rng(3)
    checked = 0
    for i in rng.choice(x.shape[1], 12, replace=False):
        xi, Di = x[:, i:i + 1], D[:, i:i + 1]
        lo, hi = oracle_lib.windows(p, xi)
        stable = True
        for a in range(3):
            for sgn in (-1, 1):
                xs = xi.copy()
                xs[a] += sgn * h
                l2, h2 = oracle_lib.windows(p, xs)
                stable &= bool(np.all(l2 == lo) and np.all(h2 == hi))
        if not stable:
            continue
        axes = [np.arange(lo[a, 0], hi[a, 0] + 1) % w.n[a] for a in range(3)]
        gz, gy, gxn = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        nodes = np.stack([gxn.ravel(), gy.ravel(), gz.ravel()])
        Sb = S_ref[:, gz.ravel(), gy.ravel(), gxn.ravel()]
        Tb = T[:, gz.ravel(), gy.ravel(), gxn.ravel()]
        own = oracle_lib.scatter_nodes(p, xi, Di, nodes)

        def local_loss(xx, DD):
            s_new = oracle_lib.scatter_nodes(p, xx, DD, nodes)
            return np.sum((Sb - own + s_new - Tb) ** 2)

        def cdiff(f, base, a, hh):
            bp, bm = base.copy(), base.copy()
            bp[a] += hh
            bm[a] -= hh
            return (f(bp) - f(bm)) / (2 * hh)

        # central differences at h and h/2 with one Richardson step (error
        # O(h^4)); errors measured against the size of the particle's
        # gradient vector, components can be small
        gscale_x = max(np.linalg.norm(rdx[:, i]), 1.0)
        gscale_D = max(np.linalg.norm(rdD[:, i]), 1.0)
        for a in range(3):
            fx = lambda xx: local_loss(xx, Di)  # noqa: E731
            f1, f2 = cdiff(fx, xi, a, h), cdiff(fx, xi, a, h / 2)
            fd = (4 * f2 - f1) / 3
            assert abs(fd - rdx[a, i]) < 1e-8 * gscale_x
            assert abs(fd - gx[a, i]) < 1e-4 * gscale_x
            fDf = lambda DD: local_loss(xi, DD)  # noqa: E731
            fd = cdiff(fDf, Di, a, h)  # quadratic in D: exact up to rounding
            assert abs(fd - rdD[a, i]) < 1e-8 * gscale_D
            assert abs(fd - gD[a, i]) < 1e-4 * gscale_D
        checked += 1
    assert checked >= 8

"""Seeded random configurations of the coupling step against the oracle.

Twelve fixed seeds draw a grid (20-72 nodes per axis, unequal), a box with
unequal spacings, sigma_R / dx between 1 and 2.4 (windows of 7-15 nodes), a
cutoff between 2.5 and 3.5, a particle cloud (uniform or clustered, 50-2500
particles), a mean shear and gravity.  For each: integer stencil windows bit
for bit, and three coupled steps (the first without removal) with the source,
force and velocity within 1e-5 (FP32, relative L2) and 1e-12 (FP64); then the
options (PIC, point-value gather, delayed source, general force) on six of
them, five steps each against their oracle steps.
"""

import dataclasses
import math

import numpy as np
import pytest

import erpp_inputs as I
from test_gpu_full_force import _fp32_bound

pytestmark = pytest.mark.gpu

SEEDS = list(range(12))


@pytest.fixture(scope="module")
def erpp(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_6969_gb300 as pkg
    return pkg


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    n = tuple(int(v) for v in rng.integers(20, 73, 3))
    dx = 2 * math.pi / 48 * rng.uniform(0.8, 1.25, 3)          # unequal spacings
    L = tuple(float(n[a] * dx[a]) for a in range(3))
    sod = float(rng.uniform(1.0, 2.4))
    cutoff = float(rng.uniform(2.5, 3.5))
    # sigma_R from the largest spacing: every axis keeps at least one node of reach
    sigma = sod * float(dx.max())
    # the FP32 tiles take windows of at most 16 nodes per axis
    cutoff = min(cutoff, 7.4 * float(dx.min()) / sigma)
    cloud = "clusters" if rng.uniform() < 0.5 else "uniform"
    npart = int(rng.integers(50, 2501))
    w = dataclasses.replace(I.CFG_SMALL, name=f"fuzz{seed}", n=n, L=L, n_particles=npart,
                            sigma_over_dx=sigma / (L[0] / n[0]), cutoff=cutoff,
                            cloud=cloud, cluster_std=0.4, kmax=3.0,
                            shear_rate=float(rng.uniform(-1, 1)), field_seed=seed,
                            particle_seed=seed)
    g = tuple(float(v) for v in rng.normal(0, 2, 3))
    return w, g


def _valid(w):
    sig = w.sigma_R
    rc = w.cutoff * sig
    return all(2 * rc < w.L[a] and rc * w.n[a] / w.L[a] >= 1.0 for a in range(3))


@pytest.mark.parametrize("seed", SEEDS)
def test_fuzz_windows_and_steps(erpp, oracle_lib, seed):
    w, g = _config(seed)
    if not _valid(w):
        pytest.skip("drawn parameters outside the library's stencil limits")
    p = w.params(gravity=g)
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    ctx32 = erpp.Context(p, precision="fp32")
    lo, hi = ctx32.debug_windows(cuda(st.x))
    rlo, rhi = oracle_lib.windows(p, st.x)
    assert np.array_equal(lo.cpu().numpy(), rlo) and np.array_equal(hi.cpu().numpy(), rhi)
    for precision, tol in (("fp32", 1e-5), ("fp64", 1e-12)):
        import torch
        ctx = ctx32 if precision == "fp32" else erpp.Context(p, precision="fp64")
        dtype = torch.float32 if precision == "fp32" else torch.float64
        ps = erpp.ParticleState.from_numpy(st)
        u = cuda(grid, dtype)
        S = ctx.new_grid()
        ref = st.copy()
        for k in range(3):
            ctx.step(u, ps, S=S, first_step=(k == 0))
            S_ref = oracle_lib.step(p, grid, ref, first_step=(k == 0))
            assert rel(S.cpu().numpy(), S_ref) < tol, (precision, k)
            assert rel(ps.D.cpu().numpy(), ref.D) < tol, (precision, k)
            assert rel(ps.v.cpu().numpy(), ref.v) < tol, (precision, k)
        ctx.check()


KINDS = ("pic", "point", "lag", "full")


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("kind", KINDS)
def test_fuzz_options(erpp, oracle_lib, kind, seed):
    """The options on the same random configurations, five steps each against
    their oracle steps: PIC and point-value weights, the source delayed by
    L = 2 steps (dt = eps_R / 2 with nu = 1 and particles of radius 0.05, so
    that the step stays short and stable), the general force (rho_p / rho_f =
    2, radius 0.05; in FP32 within the bound that the one-step differences of
    u~ set on the gather's rounding, as in the general-force parity tests)."""
    import torch
    from oracle import full_force as FF
    from oracle import lagged as LG
    from oracle import weights as W
    w, g = _config(seed)
    if not _valid(w):
        pytest.skip("drawn parameters outside the library's stencil limits")
    if kind == "lag":
        # dt = eps_R / 2: nu = 1 keeps eps_R (and the step) short, radius 0.05
        # keeps tau_p above dt
        w = dataclasses.replace(w, radius=0.05, nu=1.0)
        p = w.params(gravity=g, dt=w.eps_R / 2.0)
    elif kind == "full":
        w = dataclasses.replace(w, radius=0.05, rho_ratio=2.0)
        p = w.params(gravity=g)
    else:
        p = w.params(gravity=g)
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    opts = {"pic": dict(weights="pic"), "point": dict(weights="point"),
            "lag": dict(lag=True), "full": dict(full_force=True)}[kind]
    for precision in ("fp32", "fp64"):
        tol = 1e-5 if precision == "fp32" else 1e-11
        dtype = torch.float32 if precision == "fp32" else torch.float64
        ctx = erpp.Context(p, precision=precision, **opts)
        ps = erpp.ParticleState.from_numpy(st)
        u = cuda(grid, dtype)
        S = ctx.new_grid()
        ref, hist = st.copy(), (LG.History() if kind == "lag" else FF.History())
        for k in range(5):
            first = k == 0
            ctx.step(u, ps, S=S, first_step=first)
            if kind in ("pic", "point"):
                S_ref = W.step(p, grid, ref, kind, first_step=first)
            elif kind == "lag":
                S_ref = LG.step(p, grid, ref, hist, first_step=first)
            else:
                S_ref = FF.step(p, grid, ref, hist, first_step=first)
                if precision == "fp32" and not first:
                    tol = _fp32_bound(p, st, hist.ut, ref.D)
            got = S.cpu().numpy()
            if np.abs(S_ref).max() == 0.0:
                assert float(np.abs(got).max()) == 0.0, (precision, k)
            else:
                assert rel(got, S_ref) < tol, (precision, k)
            assert rel(ps.D.cpu().numpy(), ref.D) < tol, (precision, k)
            assert rel(ps.v.cpu().numpy(), ref.v) < tol, (precision, k)
        ctx.check()

"""GPU test of the host-data step (erpp_step_host through Context.step_host).

Several calls are issued back to back (their copies and steps overlap), each
with its own host field and source buffer; the results must equal those of
the device-resident step run from the same initial state, step by step.
"""

import dataclasses
import math

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def erpp():
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


CASES = [
    ("cube32", I.CFG_SMALL, "fp32"),
    ("ragged_72x40x20", dataclasses.replace(I.CFG_CLUSTERED, n=(72, 40, 20), n_particles=3000,
                                            cluster_std=0.3, kmax=3.0), "fp32"),
    ("cube32_fp64", I.CFG_SMALL, "fp64"),
]


@pytest.mark.parametrize("name,w,precision", CASES, ids=[c[0] for c in CASES])
def test_host_step_matches_device_step(erpp, name, w, precision):
    import torch
    dt = torch.float32 if precision == "fp32" else torch.float64
    grids = []
    for k in range(3):
        g, _ = I.make_grid(dataclasses.replace(w, field_seed=w.field_seed + k))
        grids.append(g)
    st = I.make_particles(w, None)
    p = w.params(gravity=(0.0, -9.81, 0.0))
    tol = 1e-6 if precision == "fp32" else 1e-13
    # device-resident reference, step by step
    ctx_d = erpp.Context(p, precision=precision)
    ps = erpp.ParticleState.from_numpy(st)
    S_dev, P_dev = [], []
    for k in range(3):
        S = ctx_d.step(torch.as_tensor(grids[k], dtype=dt).cuda(), ps, first_step=(k == 0))
        S_dev.append(S.cpu().numpy().copy())
        P_dev.append({a: getattr(ps, a).cpu().numpy().copy() for a in ("x", "v", "x_prev", "D")})
    ctx_d.check()
    # host data, three calls in flight
    ctx_h = erpp.Context(p, precision=precision)
    hst = erpp.ParticleState.from_numpy(st).pinned()
    hu = [torch.as_tensor(g, dtype=dt).pin_memory() for g in grids]
    hS = [torch.empty(g.shape, dtype=dt).pin_memory() for g in grids]
    snaps = []
    for k in range(3):
        ctx_h.step_host(hu[k], hst, hS[k], first_step=(k == 0))
    ctx_h.step_host_wait()
    torch.cuda.synchronize()
    ctx_h.check()
    for k in range(3):
        assert rel(hS[k].numpy(), S_dev[k]) < tol, (name, k)
    for a in ("x", "v", "x_prev", "D"):
        assert rel(getattr(hst, a).numpy(), P_dev[2][a]) < tol, (name, a)


def test_host_step_rejects_device_tensors(erpp):
    import torch
    w = I.CFG_SMALL
    ctx = erpp.Context(w.params())
    ps = erpp.ParticleState.from_numpy(I.make_particles(w, None))
    u = ctx.new_grid()
    with pytest.raises(TypeError):
        ctx.step_host(u, ps, u)

"""The allocation-free gather entry point, checked against erpp_interpolate.

erpp_interpolate_noalloc serves callers that must not allocate device
memory; it reuses one fixed scratch array in the library image.  Called
twice in a row through the C ABI, it must return what the context-based
erpp_interpolate returns, within the FP32 parity tolerance, both in a fresh
process and after the other tests.
"""

import ctypes

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_interpolate_matches_context_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6969_gb300 import Context, _lib
    from paper_1405_6969_gb300.erpp import _vec3

    # isotropic spacing (sigma_R = dx on every axis), tiles with ragged edges
    w = I.CFG_SMALL.scaled("noalloc", (72, 40, 20), 3000,
                           L=(2 * np.pi, 2 * np.pi * 40 / 72, 2 * np.pi * 20 / 72))
    p = w.params()
    grid, field = I.make_grid(w)
    u = torch.as_tensor(grid, dtype=torch.float32).cuda().contiguous()
    lib = _lib.load()
    prm = _lib.Params()
    prm.nx, prm.ny, prm.nz = w.n
    prm.Lx, prm.Ly, prm.Lz = w.L
    prm.nu, prm.rho_f, prm.eps_R, prm.cutoff, prm.dt = w.nu, w.rho_f, w.eps_R, w.cutoff, w.dt
    prm.gravity = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    prm.shear_rate = w.shear_rate
    prm.flags = _lib.FP32 | _lib.NORMALIZE | _lib.SELF_REMOVAL
    ctx = Context(p, precision="fp32")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):  # two calls in a row, different clouds
        x = torch.as_tensor(I.uniform_positions(3000, w.L, seed)).cuda().contiguous()
        ref = ctx.interpolate(u, x)
        out = torch.full((3, 3000), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.erpp_interpolate_noalloc(ctypes.byref(prm), ctypes.c_void_p(u.data_ptr()),
                                          3000, _vec3(x), _vec3(out), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    # beyond the stated maximum: rejected before any launch
    big = torch.zeros((3, 40000), dtype=torch.float64, device="cuda")
    assert lib.erpp_interpolate_noalloc(ctypes.byref(prm), ctypes.c_void_p(u.data_ptr()),
                                        40000, _vec3(big), _vec3(big), stream) == 1
    ctx.close()

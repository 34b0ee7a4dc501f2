"""The allocation-free gather entry point, checked against erpp_interpolate.

erpp_interpolate_noalloc serves callers that must not allocate device
memory (a frozen or exhausted memory pool, a plugin with a fixed device
budget); it reuses one fixed scratch array in the library image.  Called
twice in a row through the C ABI, it must return what the context-based
erpp_interpolate returns, within the FP32 parity tolerance, for both tile
designs and near its stated limits (16384 particles, 131072 pieces, 4096
tiles).  The first case also runs in a fresh process of its own, where the
first call looks up the array's address.
"""

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import erpp_inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# (name, grid, box, particles): isotropic spacing so that sigma_R = dx on
# every axis unless stated
CASES = [
    # x/y-halo tiles with ragged edges
    ("xy_halo_72x40x20", (72, 40, 20), (2 * np.pi, 2 * np.pi * 40 / 72, 2 * np.pi * 20 / 72), 3000),
    # y spacing a third of x: windows of 19 nodes in y, x-halo tiles cut in y and z
    ("x_halo_32x96x24", (32, 96, 24), (2 * np.pi,) * 3, 1500),
    # the stated limits: 16384 particles, 4096 tiles, 98304 pieces
    ("limits_512x256x128", (512, 256, 128), (4 * np.pi, 2 * np.pi, np.pi), 16384),
]


def check_case(name, n, L, npart):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6969_gb300 import Context, _lib
    from paper_1405_6969_gb300.erpp import _vec3

    w = I.CFG_SMALL.scaled("noalloc_" + name, n, npart, L=L)
    p = w.params()
    grid, _ = I.make_grid(w, kmax=3.0)
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
        x = torch.as_tensor(I.uniform_positions(npart, w.L, seed)).cuda().contiguous()
        ref = ctx.interpolate(u, x)
        out = torch.full((3, npart), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.erpp_interpolate_noalloc(ctypes.byref(prm), ctypes.c_void_p(u.data_ptr()),
                                          npart, _vec3(x), _vec3(out), stream)
        assert st == 0, (name, st)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5, name
    # beyond the stated maximum: rejected before any launch
    big = torch.zeros((3, 40000), dtype=torch.float64, device="cuda")
    assert lib.erpp_interpolate_noalloc(ctypes.byref(prm), ctypes.c_void_p(u.data_ptr()),
                                        40000, _vec3(big), _vec3(big), stream) == 1
    ctx.close()


@pytest.mark.parametrize("name,n,L,npart", CASES, ids=[c[0] for c in CASES])
def test_noalloc_interpolate_matches_context_path(name, n, L, npart):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    check_case(name, n, L, npart)


def test_noalloc_in_a_fresh_process():
    """The first case in a process of its own: its first call looks up the
    array's device address in a context that has made no other call."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    name, n, L, npart = CASES[0]
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "from test_zz_no_alloc import check_case; check_case(%r, %r, %r, %r); print('ok')"
            % (ROOT, os.path.join(ROOT, "tests"), name, n, L, npart))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr

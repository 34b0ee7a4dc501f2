"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point that include/erpp.h declares, and rejects
invalid parameters before touching the device."""

import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1405_6969_gb300 import _lib, build
    build.build()
    return _lib


def test_exports_every_declared_symbol(lib):
    import subprocess
    names = lib.header_symbols()
    assert {"erpp_init", "erpp_interpolate", "erpp_particle_advance", "erpp_scatter_source",
            "erpp_step", "erpp_momentum", "erpp_destroy", "erpp_status_string"} <= set(names)
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def _params(lib, **kw):
    p = lib.Params()
    p.nx = p.ny = p.nz = 32
    p.Lx = p.Ly = p.Lz = 6.283185307179586
    p.nu, p.rho_f, p.cutoff, p.dt = 0.01, 1.0, 3.0, 1e-3
    p.eps_R = (6.283185307179586 / 32) ** 2 / 0.02
    p.flags = lib.FP32 | lib.NORMALIZE | lib.SELF_REMOVAL
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(Lx=-1.0), dict(nu=0.0), dict(eps_R=float("nan")), dict(cutoff=0.0),
    dict(cutoff=40.0), dict(flags=0), dict(flags=3), dict(flags=2 | 16), dict(flags=1 | 512),
    dict(flags=1 | 8 | 32), dict(flags=1 | 32 | 64), dict(flags=1 | 16 | 32),
    dict(flags=1 | 32 | 128), dict(flags=1 | 64 | 128), dict(flags=1 | 128, dt=0.0),
    dict(flags=1 | 128 | 256), dict(flags=1 | 32 | 256), dict(flags=1 | 256, dt=0.0),
    dict(dt=-1.0), dict(rho_f=0.0)])
def test_init_rejects_invalid(lib, bad):
    so = lib.load()
    h = ctypes.c_void_p(1234)
    st = so.erpp_init(ctypes.byref(_params(lib, **bad)), ctypes.byref(h))
    assert st == 1  # ERPP_EINVAL, before any CUDA call
    assert not h.value


def test_null_arguments(lib):
    so = lib.load()
    assert so.erpp_init(None, None) == 1
    assert so.erpp_destroy(None) == 0
    assert so.erpp_step(None, None, None, None, 0, None) == 1
    assert so.erpp_check(None, None) == 1
    assert so.erpp_shared_add_rate(0, None) == 1
    for s in range(8):
        assert so.erpp_status_string(s)

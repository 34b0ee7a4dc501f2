"""FP64 CPU oracle of the ERPP coupling step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never touches it.  The arithmetic lives in ``erpp_oracle.c``
(plain double-precision loops, compiled with ``-ffp-contract=off``); this
module only marshals NumPy arrays through ctypes.

Array conventions: particle vectors ``[3, n]`` float64, grid fields
``[3, nz, ny, nx]`` float64, nodes at ``x_j = j L / N``.

Sibling modules (plain NumPy on top of these functions): ``stokes`` (the
exact Stokes step of the fluid stand-in), ``validation`` (the references of
the paper's validation cases), ``weights`` (PIC and point-value weights),
``lagged`` (the source delayed by eps_R) and ``full_force`` (the general
particle force).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "erpp_oracle.c")
_LIB = os.path.join(_HERE, "liberpp_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (plain C11, -ffp-contract=off)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("normalize", ctypes.c_int32),
        ("self_removal", ctypes.c_int32),
        ("untruncated", ctypes.c_int32),
        ("L", ctypes.c_double * 3),
        ("nu", ctypes.c_double),
        ("rho_f", ctypes.c_double),
        ("eps_R", ctypes.c_double),
        ("cutoff", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("shear_rate", ctypes.c_double),
    ]


def make_params(n, L, nu, rho_f, eps_R, cutoff, dt, gravity=(0.0, 0.0, 0.0),
                shear_rate=0.0, normalize=True, self_removal=True,
                untruncated=False):
    p = Params()
    p.n = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    p.L = (ctypes.c_double * 3)(*[float(v) for v in L])
    p.nu, p.rho_f, p.eps_R = float(nu), float(rho_f), float(eps_R)
    p.cutoff, p.dt = float(cutoff), float(dt)
    p.gravity = (ctypes.c_double * 3)(*[float(v) for v in gravity])
    p.shear_rate = float(shear_rate)
    p.normalize = int(bool(normalize))
    p.self_removal = int(bool(self_removal))
    p.untruncated = int(bool(untruncated))
    return p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(Params)
            d = ctypes.POINTER(ctypes.c_double)
            i32 = ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.c_int64
            sig = {
                "orc_windows": [P, i64, d, i32, i32],
                "orc_scatter": [P, i64, d, d, d],
                "orc_gather": [P, i64, d, d, d],
                "orc_advance": [P, i64, d, d, d, d, d, d, d, ctypes.c_int],
                "orc_step": [P, i64, d, d, d, d, d, d, d, ctypes.c_int, d, d],
                "orc_momentum": [P, i64, d, d, d, d],
                "orc_scatter_backward": [P, i64, d, d, d, d, d],
                "orc_gather_backward": [P, i64, d, d, d, d, d],
                "orc_scatter_nodes": [P, i64, d, d, i64, i32, d],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.orc_self_velocity.argtypes = [P, i64, d, d, d]
            lib.orc_self_velocity.restype = None
            lib.orc_self_velocity_s2.argtypes = [P, ctypes.c_double, i64, d, d, d]
            lib.orc_self_velocity_s2.restype = None
            _lib = lib
    return _lib


def _params(p):
    return p if isinstance(p, Params) else make_params(**p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == tuple(shape), (a.shape, shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st, name):
    if st != 0:
        raise ValueError(f"{name}: oracle status {st}")


def _grid_shape(p):
    return (3, int(p.n[2]), int(p.n[1]), int(p.n[0]))


def windows(p, x):
    """Stencil windows (j_lo, j_hi), int32 [3, n] each."""
    p = _params(p)
    x = _f64(x)
    n = x.shape[1]
    lo = np.zeros((3, n), dtype=np.int32)
    hi = np.zeros((3, n), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(_load().orc_windows(ctypes.byref(p), n, _ptr(x),
                               lo.ctypes.data_as(ip), hi.ctypes.data_as(ip)),
           "windows")
    return lo, hi


def scatter(p, x, D):
    """Regularised momentum source S [3, nz, ny, nx] of forces D at x."""
    p = _params(p)
    x, D = _f64(x), _f64(D)
    S = np.empty(_grid_shape(p))
    _check(_load().orc_scatter(ctypes.byref(p), x.shape[1], _ptr(x), _ptr(D),
                               _ptr(S)), "scatter")
    return S


def gather(p, x, u):
    """Kernel gather of grid field u at positions x, plus the mean shear."""
    p = _params(p)
    x, u = _f64(x), _f64(u, _grid_shape(p))
    up = np.empty_like(x)
    _check(_load().orc_gather(ctypes.byref(p), x.shape[1], _ptr(x), _ptr(u),
                              _ptr(up)), "gather")
    return up


def self_velocity(p, r, D, s2=None):
    """Closed-form self disturbance v_self(r; D) [3, n]; by default at the
    variance the matching kernel gather sees, else at ``s2``."""
    p = _params(p)
    r, D = _f64(r), _f64(D)
    out = np.empty_like(r)
    if s2 is None:
        _load().orc_self_velocity(ctypes.byref(p), r.shape[1], _ptr(r), _ptr(D), _ptr(out))
    else:
        _load().orc_self_velocity_s2(ctypes.byref(p), float(s2), r.shape[1], _ptr(r),
                                     _ptr(D), _ptr(out))
    return out


def advance(p, up, state, first_step=False):
    """Self removal + drag + Euler step; updates ``state`` in place."""
    p = _params(p)
    up = _f64(up)
    arrs = [state.x, state.v, state.x_prev, state.D]
    for a in arrs:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(_load().orc_advance(ctypes.byref(p), state.n, _ptr(up),
                               _ptr(state.x), _ptr(state.v),
                               _ptr(state.x_prev), _ptr(state.D),
                               _ptr(_f64(state.radius)),
                               _ptr(_f64(state.rho_p)), int(bool(first_step))),
           "advance")
    return state


def step(p, u, state, first_step=False, return_up=False):
    """One coupling step (gather, removal, drag, advance, scatter) in place.

    Returns the source S (and the gathered velocity when ``return_up``)."""
    p = _params(p)
    u = _f64(u, _grid_shape(p))
    S = np.empty(_grid_shape(p))
    up = np.empty((3, state.n))
    _check(_load().orc_step(ctypes.byref(p), state.n, _ptr(u), _ptr(state.x),
                            _ptr(state.v), _ptr(state.x_prev), _ptr(state.D),
                            _ptr(_f64(state.radius)), _ptr(_f64(state.rho_p)),
                            int(bool(first_step)), _ptr(S), _ptr(up)), "step")
    return (S, up) if return_up else S


def momentum(p, x, D, S):
    """(grid momentum dV sum S, particle momentum -(1/rho_f) sum M_p D_p)."""
    p = _params(p)
    x, D, S = _f64(x), _f64(D), _f64(S, _grid_shape(p))
    out = np.empty(6)
    _check(_load().orc_momentum(ctypes.byref(p), x.shape[1], _ptr(x), _ptr(D),
                                _ptr(S), _ptr(out)), "momentum")
    return out[:3].copy(), out[3:].copy()


def scatter_backward(p, x, D, R):
    """(dL/dD, dL/dx) for the cotangent R = dL/dS."""
    p = _params(p)
    x, D, R = _f64(x), _f64(D), _f64(R, _grid_shape(p))
    dD, dx = np.empty_like(x), np.empty_like(x)
    _check(_load().orc_scatter_backward(ctypes.byref(p), x.shape[1], _ptr(x),
                                        _ptr(D), _ptr(R), _ptr(dD), _ptr(dx)),
           "scatter_backward")
    return dD, dx


def gather_backward(p, x, u, G):
    """(dL/du, dL/dx) for the cotangent G = dL/du_p."""
    p = _params(p)
    x, u, G = _f64(x), _f64(u, _grid_shape(p)), _f64(G)
    du, dx = np.empty(_grid_shape(p)), np.empty_like(x)
    _check(_load().orc_gather_backward(ctypes.byref(p), x.shape[1], _ptr(x),
                                       _ptr(u), _ptr(G), _ptr(du), _ptr(dx)),
           "gather_backward")
    return du, dx


def scatter_nodes(p, x, D, nodes):
    """Source S[3, k] at the nodes [3, k] (int, x/y/z node indices) only."""
    p = _params(p)
    x, D = _f64(x), _f64(D)
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    k = nodes.shape[1]
    out = np.empty((3, k))
    _check(_load().orc_scatter_nodes(ctypes.byref(p), x.shape[1], _ptr(x), _ptr(D), k,
                                     nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     _ptr(out)), "scatter_nodes")
    return out


def step_threads(p, u, state, nthreads, first_step=False):
    """The same step as ``step``, on ``nthreads`` host threads.

    The particles are split into contiguous chunks and each thread runs the
    unchanged oracle step on its chunk into a source of its own (the C calls
    release the interpreter lock); the partial sources are then summed by the
    threads over z-slabs.  Particle results equal those of ``step`` exactly
    (every particle is updated on its own); the source differs only in the
    order of its FP64 sums.  Used to time the oracle on all host cores."""
    import concurrent.futures as cf
    p = _params(p)
    u = _f64(u, _grid_shape(p))
    n = state.n
    nthreads = max(1, min(int(nthreads), n)) if n else 1
    cuts = [n * k // nthreads for k in range(nthreads + 1)]
    names = ("x", "v", "x_prev", "D", "radius", "rho_p")
    chunks = []
    for k in range(nthreads):
        a, b = cuts[k], cuts[k + 1]
        chunks.append(type(state)(*(np.ascontiguousarray(getattr(state, m)[..., a:b])
                                    for m in names)))
    with cf.ThreadPoolExecutor(nthreads) as ex:
        parts = list(ex.map(lambda c: step(p, u, c, first_step=first_step), chunks))
        S = parts[0]
        nz = S.shape[1]
        zc = [nz * k // nthreads for k in range(nthreads + 1)]

        def reduce_slab(k):
            sl = slice(zc[k], zc[k + 1])
            for part in parts[1:]:
                np.add(S[:, sl], part[:, sl], out=S[:, sl])

        list(ex.map(reduce_slab, range(nthreads)))
    for k, c in enumerate(chunks):
        a, b = cuts[k], cuts[k + 1]
        for m in ("x", "v", "x_prev", "D"):
            getattr(state, m)[..., a:b] = getattr(c, m)
    return S

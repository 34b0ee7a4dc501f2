"""PyTorch binding of the ERPP C ABI.

PyTorch supplies device memory and the current CUDA stream; every step of
the coupling runs in the CUDA kernels of ``liberpp.so``.  Tensors are
passed by data pointer: particle vectors are ``[3, n]`` float64 CUDA tensors
(component-major, contiguous), grid fields ``[3, nz, ny, nx]`` float32
(``precision="fp32"``) or float64 (``precision="fp64"``).
"""

from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib


def _dptr(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), _lib._dp)


def _require_host(t, dtype, ndim):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a host (CPU) tensor")
    if t.dtype != dtype or t.dim() != ndim or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor of rank {ndim}, "
                        f"got {t.dtype} {tuple(t.shape)}")


def _vec3(t, host=False):
    """[3, n] float64 CUDA (or, host=True, CPU) tensor -> double*[3]."""
    (_require_host if host else _require)(t, torch.float64, 2)
    assert t.shape[0] == 3
    n = t.shape[1]
    base = t.data_ptr()
    return _lib._dp3(*[ctypes.cast(ctypes.c_void_p(base + 8 * n * c), _lib._dp)
                       for c in range(3)])


def _require(t, dtype, ndim):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or t.dim() != ndim or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor of rank {ndim}, "
                        f"got {t.dtype} {tuple(t.shape)}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class ParticleState:
    """Particle arrays on the device: x, v, x_prev, D are [3, n] float64;
    radius and rho_p are [n] float64."""

    x: torch.Tensor
    v: torch.Tensor
    x_prev: torch.Tensor
    D: torch.Tensor
    radius: torch.Tensor
    rho_p: torch.Tensor

    @property
    def n(self):
        return self.x.shape[1]

    @staticmethod
    def from_numpy(st, device="cuda"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float64).contiguous().to(device)  # noqa: E731
        return ParticleState(f(st.x), f(st.v), f(st.x_prev), f(st.D), f(st.radius),
                             f(st.rho_p))

    def to_c(self, host=False):
        """erpp_particles of the arrays (CUDA tensors; CPU ones with host=True)."""
        P = _lib.Particles()
        P.n = self.n
        P.x, P.v = _vec3(self.x, host), _vec3(self.v, host)
        P.x_prev, P.D = _vec3(self.x_prev, host), _vec3(self.D, host)
        req = _require_host if host else _require
        req(self.radius, torch.float64, 1)
        req(self.rho_p, torch.float64, 1)
        P.radius, P.rho_p = _dptr(self.radius), _dptr(self.rho_p)
        return P

    def pinned(self):
        """Copy of the state in page-locked host memory."""
        return ParticleState(*(t.detach().cpu().pin_memory() for t in
                               (self.x, self.v, self.x_prev, self.D, self.radius, self.rho_p)))


WEIGHTS = ("gaussian", "pic", "point")


def make_params(params, precision="fp32", normalize=True, self_removal=True, kahan=False,
                weights="gaussian", lag=False, full_force=False):
    """erpp_params from a parameter dict (n, L, nu, rho_f, eps_R, cutoff, dt,
    gravity, shear_rate) and the option flags.  ``weights``: "gaussian" (the
    regularised kernel and its matching gather), "pic" (trilinear projection
    and interpolation, no self removal) or "point" (Gaussian source, 4-point
    Lagrange point-value gather).  ``lag``: delay the source of erpp_step by
    eps_R (round(eps_R / dt) steps, the literal Eq. ns_regularized_filtered).
    ``full_force``: the general force of Eq. force_particle (Faxen, added mass,
    one-step Basset memory) instead of the Stokes drag."""
    if weights not in WEIGHTS:
        raise ValueError(f"weights must be one of {WEIGHTS}")
    p = _lib.Params()
    p.nx, p.ny, p.nz = (int(v) for v in params["n"])
    p.Lx, p.Ly, p.Lz = (float(v) for v in params["L"])
    p.nu, p.rho_f = float(params["nu"]), float(params.get("rho_f", 1.0))
    p.eps_R, p.cutoff = float(params["eps_R"]), float(params["cutoff"])
    p.dt = float(params["dt"])
    p.gravity = (ctypes.c_double * 3)(*[float(g) for g in params.get("gravity", (0, 0, 0))])
    p.shear_rate = float(params.get("shear_rate", 0.0))
    flags = {"fp32": _lib.FP32, "fp64": _lib.FP64}[precision]
    if normalize:
        flags |= _lib.NORMALIZE
    if self_removal:
        flags |= _lib.SELF_REMOVAL
    if kahan:
        flags |= _lib.KAHAN
    if weights == "pic":
        flags |= _lib.PIC
    elif weights == "point":
        flags |= _lib.POINT_GATHER
    if lag:
        flags |= _lib.LAG
    if full_force:
        flags |= _lib.FULL_FORCE
    p.flags = flags
    return p


class Context:
    """One ERPP context (grid, parameters, scratch) on the current device.

    params: dict with n=(nx, ny, nz), L=(Lx, Ly, Lz), nu, rho_f, eps_R,
    cutoff, dt, gravity=(gx, gy, gz), shear_rate.  weights: "gaussian" (the
    ERPP kernel), "pic" (trilinear particle-in-cell coupling, no self
    removal) or "point" (Gaussian source, 4-point Lagrange point-value
    gather); see make_params.  lag: the source of step() is delayed by eps_R
    (round(eps_R / dt) steps; the context keeps the positions and forces of
    the steps in between).  full_force: step() with the general force of
    Eq. force_particle (Faxen, added mass, one-step Basset memory).
    """

    def __init__(self, params, precision="fp32", normalize=True, self_removal=True,
                 kahan=False, weights="gaussian", lag=False, full_force=False):
        self.lib = _lib.load()
        if weights == "pic":
            self_removal = False  # PIC has no closed-form self disturbance
        p = make_params(params, precision, normalize, self_removal, kahan, weights, lag,
                        full_force)
        self.weights = weights
        self.lag = bool(lag)
        self.full_force = bool(full_force)
        self.params = dict(params)
        self.precision = precision
        self.kahan = bool(kahan)
        self.grid_dtype = torch.float32 if precision == "fp32" else torch.float64
        self.shape = (3, p.nz, p.ny, p.nx)
        h = ctypes.c_void_p()
        _lib.check(self.lib.erpp_init(ctypes.byref(p), ctypes.byref(h)), "erpp_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.erpp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _grid(self, g):
        _require(g, self.grid_dtype, 4)
        if tuple(g.shape) != self.shape:
            raise ValueError(f"grid shape {tuple(g.shape)} != {self.shape}")
        return ctypes.c_void_p(g.data_ptr())

    def new_grid(self):
        return torch.empty(self.shape, dtype=self.grid_dtype, device="cuda")

    def interpolate(self, u, x, out=None, stream=None):
        n = x.shape[1]
        out = torch.empty((3, n), dtype=torch.float64, device=x.device) if out is None else out
        _lib.check(self.lib.erpp_interpolate(self._h, self._grid(u), n, _vec3(x), _vec3(out),
                                             _stream(stream)), "erpp_interpolate")
        return out

    def particle_advance(self, up, state, first_step=False, stream=None):
        P = state.to_c()
        _lib.check(self.lib.erpp_particle_advance(self._h, _vec3(up), ctypes.byref(P),
                                                  int(bool(first_step)), _stream(stream)),
                   "erpp_particle_advance")
        return state

    def scatter_source(self, x, D, S=None, stream=None):
        S = self.new_grid() if S is None else S
        _lib.check(self.lib.erpp_scatter_source(self._h, x.shape[1], _vec3(x), _vec3(D),
                                                self._grid(S), _stream(stream)),
                   "erpp_scatter_source")
        return S

    def scatter_backward(self, x, D, R, need_dD=True, stream=None):
        """(dL/dD or None, dL/dx) for the cotangent R = dL/dS of the source."""
        n = x.shape[1]
        dx = torch.empty((3, n), dtype=torch.float64, device=x.device)
        dD = torch.empty((3, n), dtype=torch.float64, device=x.device) if need_dD else None
        pdD = ctypes.byref(_vec3(dD)) if need_dD else None
        _lib.check(self.lib.erpp_scatter_backward(self._h, n, _vec3(x), _vec3(D), self._grid(R),
                                                  pdD, ctypes.byref(_vec3(dx)),
                                                  _stream(stream)), "erpp_scatter_backward")
        return dD, dx

    def gather_backward(self, x, u, g, need_du=True, need_dx=True, stream=None):
        """(dL/du or None, dL/dx or None) for the cotangent g = dL/du_p."""
        n = x.shape[1]
        du = self.new_grid() if need_du else None
        dx = torch.empty((3, n), dtype=torch.float64, device=x.device) if need_dx else None
        pdx = ctypes.byref(_vec3(dx)) if need_dx else None
        _lib.check(self.lib.erpp_gather_backward(
            self._h, n, _vec3(x), self._grid(u), _vec3(g),
            self._grid(du) if need_du else None, pdx, _stream(stream)), "erpp_gather_backward")
        return du, dx

    def step(self, u, state, S=None, first_step=False, stream=None):
        S = self.new_grid() if S is None else S
        P = state.to_c()
        _lib.check(self.lib.erpp_step(self._h, self._grid(u), ctypes.byref(P), self._grid(S),
                                      int(bool(first_step)), _stream(stream)), "erpp_step")
        return S

    def step_host(self, u, state, S, first_step=False, stream=None):
        """erpp_step_host: u, S and the ParticleState on the host (CPU tensors,
        page-locked for overlap, e.g. state.pinned()).  Returns once the copies
        and the step are enqueued; call step_host_wait() and synchronise the
        stream before reading S or the state."""
        for g in (u, S):
            _require_host(g, self.grid_dtype, 4)
            if tuple(g.shape) != self.shape:
                raise ValueError(f"grid shape {tuple(g.shape)} != {self.shape}")
        P = state.to_c(host=True)
        _lib.check(self.lib.erpp_step_host(self._h, ctypes.c_void_p(u.data_ptr()), ctypes.byref(P),
                                           ctypes.c_void_p(S.data_ptr()),
                                           int(bool(first_step)), _stream(stream)),
                   "erpp_step_host")
        return S

    def step_host_wait(self, stream=None):
        """Makes the stream wait for every step_host call so far."""
        _lib.check(self.lib.erpp_step_host_wait(self._h, _stream(stream)), "erpp_step_host_wait")

    def momentum(self, S, x, D, stream=None):
        out = (ctypes.c_double * 6)()
        _lib.check(self.lib.erpp_momentum(self._h, self._grid(S), x.shape[1], _vec3(x),
                                          _vec3(D), ctypes.cast(out, _lib._dp),
                                          _stream(stream)), "erpp_momentum")
        return list(out[:3]), list(out[3:])

    def check(self, stream=None):
        _lib.check(self.lib.erpp_check(self._h, _stream(stream)), "erpp_check")

    def set_tiling(self, tile_y=0, tile_z=0, threads=0):
        """Request T_y, T_z and threads per block of the x/y-halo tiles
        (0 = default)."""
        _lib.check(self.lib.erpp_set_tiling(self._h, int(tile_y), int(tile_z), int(threads)),
                   "erpp_set_tiling")

    def set_scatter_mode(self, mode="merge"):
        """How the FP32 scatter adds tile halos to the neighbours: "merge"
        (halo strips and two merge kernels, the default) or "cluster" (the
        x-halo through thread-block clusters, the y-halo through strips)."""
        _lib.check(self.lib.erpp_set_scatter_mode(self._h, _lib.SCATTER_MODES[mode]),
                   "erpp_set_scatter_mode")
        self._scatter_mode = mode

    def scatter_mode(self):
        return getattr(self, "_scatter_mode", "merge")

    def tiling(self):
        """(design, W, T_y, T_z, threads) of the tiles in use."""
        out = (ctypes.c_int32 * 5)()
        _lib.check(self.lib.erpp_get_tiling(self._h, out), "erpp_get_tiling")
        return tuple(int(v) for v in out)

    def last_step_launches(self):
        """Kernels the most recent step launched."""
        n = ctypes.c_int32(0)
        _lib.check(self.lib.erpp_last_step_launches(self._h, ctypes.byref(n)),
                   "erpp_last_step_launches")
        return int(n.value)

    def profile_enable(self, enable=True):
        _lib.check(self.lib.erpp_profile_enable(self._h, int(bool(enable))),
                   "erpp_profile_enable")

    def profile_read(self):
        """(milliseconds per phase [bin, gather, advance, scatter], steps)."""
        ms = (ctypes.c_double * 4)()
        n = ctypes.c_int64()
        _lib.check(self.lib.erpp_profile_read(self._h, ctypes.cast(ms, _lib._dp),
                                              ctypes.byref(n)), "erpp_profile_read")
        return list(ms), int(n.value)

    def debug_set_wait(self, limit_ns=0, stall=False):
        """Limit (nanoseconds, 0 = default) of the gather's bounded wait for its
        staged tile; ``stall`` makes the wait run out on purpose (tests of the
        ERPP_ETIMEOUT path)."""
        _lib.check(self.lib.erpp_debug_set_wait(self._h, int(limit_ns), int(bool(stall))),
                   "erpp_debug_set_wait")

    def debug_windows(self, x, stream=None):
        n = x.shape[1]
        lo = torch.empty((3, n), dtype=torch.int32, device=x.device)
        hi = torch.empty((3, n), dtype=torch.int32, device=x.device)
        _lib.check(self.lib.erpp_debug_windows(self._h, n, _vec3(x),
                                               ctypes.c_void_p(lo.data_ptr()),
                                               ctypes.c_void_p(hi.data_ptr()),
                                               _stream(stream)), "erpp_debug_windows")
        return lo, hi


class StokesFluid:
    """The fluid stand-in (erpp_fluid_*): exact periodic unsteady-Stokes
    steps forced by the source, u <- exp(-nu k^2 dt) P (u + dt S)."""

    def __init__(self, params, precision="fp32"):
        self.lib = _lib.load()
        p = make_params(params, precision)
        self.grid_dtype = torch.float32 if precision == "fp32" else torch.float64
        self.shape = (3, p.nz, p.ny, p.nx)
        h = ctypes.c_void_p()
        _lib.check(self.lib.erpp_fluid_init(ctypes.byref(p), ctypes.byref(h)), "erpp_fluid_init")
        self._h = h

    def step(self, u, S, stream=None):
        for g in (u, S):
            _require(g, self.grid_dtype, 4)
            if tuple(g.shape) != self.shape:
                raise ValueError(f"grid shape {tuple(g.shape)} != {self.shape}")
        _lib.check(self.lib.erpp_fluid_stokes_step(self._h, ctypes.c_void_p(u.data_ptr()),
                                                   ctypes.c_void_p(S.data_ptr()),
                                                   _stream(stream)), "erpp_fluid_stokes_step")
        return u

    def close(self):
        if getattr(self, "_h", None):
            self.lib.erpp_fluid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent boxes stepped together (erpp_batch_*).

    boxes: list of (params dict, u grid, ParticleState, S grid); every box
    uses the same precision and options.  The tensors must stay alive and in
    place for the batch's lifetime (the batch keeps their addresses)."""

    def __init__(self, boxes, precision="fp32", normalize=True, self_removal=True,
                 kahan=False):
        self.lib = _lib.load()
        dtype = torch.float32 if precision == "fp32" else torch.float64
        arr = (_lib.BoxDesc * len(boxes))()
        self._keep = []
        for i, (params, u, state, S) in enumerate(boxes):
            shape = (3, int(params["n"][2]), int(params["n"][1]), int(params["n"][0]))
            for g in (u, S):
                _require(g, dtype, 4)
                if tuple(g.shape) != shape:
                    raise ValueError(f"box {i}: grid shape {tuple(g.shape)} != {shape}")
            arr[i].params = make_params(params, precision, normalize, self_removal, kahan)
            arr[i].u = ctypes.c_void_p(u.data_ptr())
            arr[i].S = ctypes.c_void_p(S.data_ptr())
            arr[i].particles = state.to_c()
            self._keep.append((u, state, S))
        h = ctypes.c_void_p()
        _lib.check(self.lib.erpp_batch_init(len(boxes), arr, ctypes.byref(h)), "erpp_batch_init")
        self._h = h
        self._opts = dict(precision=precision, normalize=normalize, self_removal=self_removal,
                          kahan=kahan)
        self._boxes = list(boxes)

    def set_tiling(self, box, tile_y=0, tile_z=0, threads=0):
        _lib.check(self.lib.erpp_batch_set_tiling(self._h, int(box), int(tile_y), int(tile_z),
                                                  int(threads)), "erpp_batch_set_tiling")

    BATCH_FORMS = {"branches": 0, "multi": 1}

    def set_form(self, form="branches"):
        """The graph's form: one branch per box ("branches") or nine kernels
        over all boxes ("multi", erpp_batch_set_form)."""
        _lib.check(self.lib.erpp_batch_set_form(self._h, self.BATCH_FORMS[form]),
                   "erpp_batch_set_form")

    def last_step_launches(self):
        """Kernels of one batched step (the boxes' most recent step sequences,
        the ones a captured graph replays)."""
        n = ctypes.c_int32(0)
        _lib.check(self.lib.erpp_batch_last_step_launches(self._h, ctypes.byref(n)),
                   "erpp_batch_last_step_launches")
        return int(n.value)

    def tiling(self, box):
        """erpp_get_tiling of one box: (design, W, T_y, T_z, threads)."""
        out = (ctypes.c_int32 * 5)()
        _lib.check(self.lib.erpp_batch_get_tiling(self._h, int(box), out),
                   "erpp_batch_get_tiling")
        return tuple(int(v) for v in out)

    def autotune(self, steps=3, warmup=1, cache_path=None, use_cache=True):
        """Tile shape per box: each box is tuned on a stand-alone context with
        its own data (the autotuner's cache shares results between boxes of
        the same class) and the choice is applied to the batch.  Returns the
        chosen (T_y, T_z, threads) per box."""
        from . import autotune
        chosen = []
        for i, (params, u, state, _S) in enumerate(self._boxes):
            ctx = Context(params, **self._opts)
            try:
                r = autotune.tune(ctx, u, state, steps=steps, warmup=warmup,
                                  cache_path=cache_path, use_cache=use_cache)
            finally:
                ctx.close()
            if r["tile"] is not None:
                self.set_tiling(i, *r["tile"])
            chosen.append(r["tile"])
        return chosen

    def step(self, first_step=False, use_graph=True, stream=None):
        _lib.check(self.lib.erpp_step_batched(self._h, int(bool(first_step)),
                                              int(bool(use_graph)), _stream(stream)),
                   "erpp_step_batched")

    def check(self, stream=None):
        _lib.check(self.lib.erpp_batch_check(self._h, _stream(stream)), "erpp_batch_check")

    def close(self):
        if getattr(self, "_h", None):
            self.lib.erpp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SHARED_ADD_KINDS = {"s32": 0, "f32": 1}


def shared_add_rate(kind="s32"):
    """Lane adds per second of the shared-memory atomic add the scatter
    accumulates with, measured on the current device with nothing else
    limiting it (erpp_shared_add_rate): "s32" the 32-bit fixed-point add,
    "f32" the FP32 add of dense tiles."""
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    _lib.check(lib.erpp_shared_add_rate(SHARED_ADD_KINDS[kind], ctypes.byref(out)),
               "erpp_shared_add_rate")
    return float(out.value)


class ScatterSource(torch.autograd.Function):
    """S = source(x, D) (Eq. ns_regularized_filtered) with its hand-written
    adjoint: ``ScatterSource.apply(ctx, x, D)`` for [3, n] float64 x and D."""

    @staticmethod
    def forward(fctx, ectx, x, D):
        fctx.ectx = ectx
        fctx.save_for_backward(x, D)
        return ectx.scatter_source(x.detach().contiguous(), D.detach().contiguous())

    @staticmethod
    def backward(fctx, gS):
        x, D = fctx.saved_tensors
        dD, dx = fctx.ectx.scatter_backward(x.detach().contiguous(), D.detach().contiguous(),
                                            gS.contiguous(),
                                            need_dD=fctx.needs_input_grad[2])
        return None, (dx if fctx.needs_input_grad[1] else None), dD


class Interpolate(torch.autograd.Function):
    """u_p = gather(u, x) with its hand-written adjoint:
    ``Interpolate.apply(ctx, u, x)`` for a grid u and [3, n] float64 x."""

    @staticmethod
    def forward(fctx, ectx, u, x):
        fctx.ectx = ectx
        fctx.save_for_backward(u, x)
        return ectx.interpolate(u.detach().contiguous(), x.detach().contiguous())

    @staticmethod
    def backward(fctx, g):
        u, x = fctx.saved_tensors
        du, dx = fctx.ectx.gather_backward(x.detach().contiguous(), u.detach().contiguous(),
                                           g.contiguous(), need_du=fctx.needs_input_grad[1],
                                           need_dx=fctx.needs_input_grad[2])
        return None, du, dx

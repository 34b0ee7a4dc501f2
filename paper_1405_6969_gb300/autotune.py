"""Tile-shape autotuner for the FP32 coupling kernels.

The FP32 gather and scatter run one thread block (256 or 512 threads) per
grid tile of W x T_y x T_z nodes (x/y-halo tiles, ``erpp_set_tiling``).
Taller tiles stage fewer halo rows per node; flatter tiles need less shared
memory (more blocks per SM) but cut more particle windows along z; more
threads per block hide more latency but split a tile's units over more
warps.  The best shape depends on the grid, the kernel width sigma_R / dx and
the particle density, so it is
measured: every candidate runs a few coupling steps (CUDA events, on copies of
the particle state), then the three fastest shapes are timed again with the
scatter's x-halo exchanged through thread-block clusters (scatter mode
"cluster") and with the x-windows cut at x-tile boundaries (scatter mode
"xclip"), and the fastest (shape, mode) is applied and remembered in a JSON
cache keyed by (grid, r_c / dx, particles per node class, options).  Host
logic only; every step it times runs in the CUDA library.
"""

from __future__ import annotations

import json
import math
import os

# (T_y, T_z, threads per block)
CANDIDATES = ((16, 4, 256), (16, 2, 256), (32, 2, 256), (32, 1, 256), (8, 4, 256),
              (16, 4, 512), (16, 2, 512), (32, 2, 512), (32, 1, 512), (8, 2, 512))


def default_cache_path():
    base = os.environ.get("ERPP_AUTOTUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "erpp", "autotune.json")


def workload_key(params, n_particles, precision="fp32", kahan=False):
    """Cache key: grid, stencil radius in grid spacings (per axis, 2 decimals),
    density class (nearest power of two of particles per node) and options."""
    n = tuple(int(v) for v in params["n"])
    L = tuple(float(v) for v in params["L"])
    sig = math.sqrt(2.0 * float(params["nu"]) * float(params["eps_R"]))
    rc = float(params["cutoff"]) * sig
    cp = tuple(round(rc * n[a] / L[a], 2) for a in range(3))
    nodes = n[0] * n[1] * n[2]
    dens = int(round(math.log2(max(n_particles, 1) / nodes))) if n_particles > 0 else -99
    return f"{n[0]}x{n[1]}x{n[2]}|cp={cp[0]},{cp[1]},{cp[2]}|d2^{dens}|{precision}|kahan={int(kahan)}"


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_steps(ctx, u, state, S, steps, warmup):
    import torch
    from .erpp import ParticleState
    ps = ParticleState(*(t.clone() for t in (state.x, state.v, state.x_prev, state.D,
                                             state.radius, state.rho_p)))
    for k in range(warmup):
        ctx.step(u, ps, S=S, first_step=(k == 0))
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ctx.step(u, ps, S=S)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    return e0.elapsed_time(e1) / steps


def tune(ctx, u, state, S=None, candidates=CANDIDATES, steps=5, warmup=2, cache_path=None,
         use_cache=True):
    """Choose and apply the fastest tile shape for this context and workload.

    Returns {"tile": (T_y, T_z, threads), "mode": scatter mode, "tiling": ctx.tiling(),
    "ms": {...} or None, "cached": bool}.  Contexts without x/y-halo tiles, PIC contexts (no tiles) and
    contexts with the delayed source (whose first round(eps_R/dt) steps have no
    source to time) are left unchanged.  Re-tiling drops the step history of a
    context with the general force: its next step must be a first step."""
    if (ctx.tiling()[0] != 4 or getattr(ctx, "weights", "gaussian") == "pic"
            or getattr(ctx, "lag", False)):
        return {"tile": None, "mode": None, "tiling": ctx.tiling(), "ms": None, "cached": False}
    path = cache_path or default_cache_path()
    key = workload_key(ctx.params, state.n, ctx.precision, getattr(ctx, "kahan", False))
    cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache and len(cache[key].get("tile", ())) == 3:
        ty, tz, nt = cache[key]["tile"]
        mode = cache[key].get("mode", "merge")
        ctx.set_tiling(ty, tz, nt)
        ctx.set_scatter_mode(mode)
        return {"tile": (ty, tz, nt), "mode": mode, "tiling": ctx.tiling(),
                "ms": cache[key].get("ms"), "cached": True}
    S = ctx.new_grid() if S is None else S
    times = {}
    ctx.set_scatter_mode("merge")
    for ty, tz, nt in candidates:
        ctx.set_tiling(ty, tz, nt)
        times[f"{ty}x{tz}x{nt}"] = _time_steps(ctx, u, state, S, steps, warmup)
    top = sorted(times, key=times.get)[:3]
    for mode in ("cluster", "xclip"):
        ctx.set_scatter_mode(mode)
        for name in top:
            ty, tz, nt = (int(v) for v in name.split("x"))
            ctx.set_tiling(ty, tz, nt)
            times[f"{name}x{mode}"] = _time_steps(ctx, u, state, S, steps, warmup)
    best = min(times, key=times.get)
    parts = best.split("x")
    ty, tz, nt = (int(v) for v in parts[:3])
    mode = parts[3] if len(parts) == 4 else "merge"
    ctx.set_tiling(ty, tz, nt)
    ctx.set_scatter_mode(mode)
    if use_cache:
        cache[key] = {"tile": [ty, tz, nt], "mode": mode, "ms": times}
        save_cache(path, cache)
    return {"tile": (ty, tz, nt), "mode": mode, "tiling": ctx.tiling(), "ms": times,
            "cached": False}

"""Measured choice of the time-step kernels' work decomposition.

For a problem shape the autotuner times candidate (tile width, height,
z blocks) decompositions of the forward kernel (tune_model) or of the
adjoint kernel (tune_gradient) with the library's own CUDA-event timing
hook over a short run, and keeps the fastest.  Results are cached in a JSON file (MAMUTE_AUTOTUNE_CACHE,
default ~/.cache/mamute/tiles.json) keyed by the padded window shape, the
number of shots, density and the kernel, and passed to the library through
the `tiles` option (the numerical result does not depend on the choice).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np

from . import mamute

SHAPES = [(64, 16), (72, 16), (48, 16), (96, 8), (64, 8), (128, 8), (32, 16), (32, 8)]
ZSPLITS = [1, 2, 3, 4, 6]


def cache_path() -> str:
    return os.environ.get("MAMUTE_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mamute", "tiles.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(c):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def key(grid, n_src, dens, kind, aperture=None):
    """Cache key of a problem.  Apertures enter through a SHA-1 digest of
    their int32 bytes, which (unlike Python's per-process salted hash of
    bytes) is the same in every process, so cached tiles are reused."""
    b = 2 * grid.border
    if aperture is None:
        ap = "full"
    else:
        raw = np.ascontiguousarray(aperture, dtype=np.int32).tobytes()
        ap = "ap" + hashlib.sha1(raw).hexdigest()[:16]
    return f"{kind}:{grid.nx + b}x{grid.ny + b}x{grid.nz + b}:s{n_src}:d{int(dens)}:{ap}"


def _timer(ctx):
    lib = ctx.lib
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.mamute_ctx_set_timing(ctx._h, 1)

    def last():
        ms, sl = ctypes.c_double(), ctypes.c_longlong()
        lib.mamute_ctx_last_timing(ctx._h, ctypes.byref(ms), ctypes.byref(sl), None)
        return ms.value / max(sl.value, 1)
    return last


def tune_model(ctx, grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, seis, aperture=None,
               steps=24, candidates=None):
    """Fastest forward decomposition for mamute_model on this problem (ms per
    step launch), cached; returns the `tiles` option to pass."""
    c = _load()
    k = key(grid, len(src_xyz), rho is not None, "fwd", aperture)
    if k in c:
        return c[k]["tiles"]
    last = _timer(ctx)
    short = mamute.make_grid(grid.nx, grid.ny, grid.nz, grid.border, grid.h, grid.dt, steps,
                             (grid.ox, grid.oy, grid.oz), grid.cerjan)
    import torch
    tmp = torch.empty((int(rec_offset[-1]), steps), device=seis.device)
    best = None
    for tx, ty in (candidates or SHAPES):
        for zs in ZSPLITS:
            tiles = [tx, ty, zs, 0, 0, 0]
            try:
                ctx.model(short, vel, rho, src_xyz, wavelet[:steps], rec_offset, rec_xyz, tmp,
                          aperture=aperture, tiles=tiles)
                ctx.model(short, vel, rho, src_xyz, wavelet[:steps], rec_offset, rec_xyz, tmp,
                          aperture=aperture, tiles=tiles)
            except mamute.MamuteError:
                continue
            t = last()
            if best is None or t < best[0]:
                best = (t, tiles)
    c = _load()
    c[k] = {"tiles": best[1], "ms_per_step": best[0]}
    _store(c)
    return best[1]


def tune_gradient(ctx, grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, d_obs, aperture=None,
                  n_snapshots=-1, steps=24, candidates=None):
    """Fastest adjoint decomposition for mamute_gradient on this problem
    (forward left to the library's cost model), timed over whole gradients
    of `steps` steps with the given storage mode, cached; returns the
    `tiles` option to pass."""
    c = _load()
    k = key(grid, len(src_xyz), rho is not None, f"adj{n_snapshots}", aperture)
    if k in c:
        return c[k]["tiles"]
    lib = ctx.lib
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.mamute_ctx_set_timing(ctx._h, 1)
    short = mamute.make_grid(grid.nx, grid.ny, grid.nz, grid.border, grid.h, grid.dt, steps,
                             (grid.ox, grid.oy, grid.oz), grid.cerjan)
    import torch
    dobs = d_obs[:, :steps].contiguous()
    grad = torch.empty_like(vel)
    best = None
    for tx, ty in (candidates or SHAPES):
        for zs in ZSPLITS:
            tiles = [0, 0, 0, tx, ty, zs]
            try:
                for _ in range(2):
                    ctx.gradient(short, vel, rho, src_xyz, wavelet[:steps], rec_offset, rec_xyz,
                                 dobs, grad, aperture=aperture, n_snapshots=n_snapshots,
                                 tiles=tiles)
            except mamute.MamuteError:
                continue
            ms = ctypes.c_double()
            lib.mamute_ctx_last_timing(ctx._h, ctypes.byref(ms), None, None)
            if best is None or ms.value < best[0]:
                best = (ms.value, tiles)
    c = _load()
    c[k] = {"tiles": best[1], "ms_per_gradient": best[0]}
    _store(c)
    return best[1]

"""ctypes front end for the FP64 oracle (mamute_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports this module.  Every function here marshals numpy arrays into the C
oracle; the arithmetic lives in mamute_oracle.cpp, which follows Eq. 1 and
Algorithms 1 and 3 of the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mamute_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (OpenMP over z planes)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("border", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("cerjan", ctypes.c_double), ("free_surface", ctypes.c_int),
                ("xyz_interp", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_grid(nx, ny, nz, border, h, dt, nt, origin=(0.0, 0.0, 0.0), cerjan=0.015,
              spacing=None, free_surface=0, xyz_interp=0) -> OGrid:
    """free_surface = 1: pressure-release top model plane (image method);
    xyz_interp = 1: trilinear sources and receivers (0: nearest node)."""
    dx, dy, dz = spacing if spacing is not None else (h, h, h)
    return OGrid(nx, ny, nz, border, dx, dy, dz, dt, nt, origin[0], origin[1], origin[2], cerjan,
                 int(free_surface), int(xyz_interp))


def padded_shape(g: OGrid):
    b = 2 * g.border
    return (g.nz + b, g.ny + b, g.nx + b)


def fd_coeffs() -> np.ndarray:
    out = np.zeros(5)
    _load().oracle_fd_coeffs(_p(out))
    return out


def prepare(g: OGrid, vel, rho=None):
    """Padded (A, m2, g, sqrt_rho) arrays, FP64."""
    shp = padded_shape(g)
    A, m2, gg, sr = (np.zeros(shp) for _ in range(4))
    vel, rho = _f64(vel), _f64(rho)
    _load().oracle_prepare(ctypes.byref(g), _p(vel), _p(rho), _p(A), _p(m2), _p(gg), _p(sr))
    return A, m2, gg, sr


def laplacian(g: OGrid, u):
    u = _f64(u)
    out = np.zeros_like(u)
    _load().oracle_laplacian(ctypes.byref(g), _p(u), _p(out))
    return out


def advance(g: OGrid, vel, uprev, ucur, n_steps, rho=None):
    """Advance (u^{-1}, u^0) -> (u^{n-1}, u^n) with no source."""
    up, uc = _f64(uprev).copy(), _f64(ucur).copy()
    vel, rho = _f64(vel), _f64(rho)
    _load().oracle_advance(ctypes.byref(g), _p(vel), _p(rho), _p(up), _p(uc), ctypes.c_int(n_steps))
    return up, uc


def _acq(src_xyz, rec_offset, rec_xyz):
    src_xyz = _f64(np.asarray(src_xyz).reshape(-1, 3))
    rec_offset = np.ascontiguousarray(rec_offset, dtype=np.int32)
    rec_xyz = _f64(np.asarray(rec_xyz).reshape(-1, 3))
    return src_xyz, rec_offset, rec_xyz


def _ap(aperture):
    return None if aperture is None else np.ascontiguousarray(aperture, dtype=np.int32)


def model(g: OGrid, vel, src_xyz, wavelet, rec_offset, rec_xyz, rho=None, precision=64,
          phess=False, aperture=None):
    """Seismograms [total_rec][nt] (FP64 array); with phess=True also the
    pseudo-Hessian [nz][ny][nx]."""
    src_xyz, rec_offset, rec_xyz = _acq(src_xyz, rec_offset, rec_xyz)
    vel, rho, wavelet = _f64(vel), _f64(rho), _f64(wavelet)
    seis = np.zeros((int(rec_offset[-1]), g.nt))
    ph = np.zeros((g.nz, g.ny, g.nx)) if phess else None
    ap = _ap(aperture)
    rc = _load().oracle_model(ctypes.byref(g), _p(vel), _p(rho), ctypes.c_int(len(src_xyz)),
                              _p(src_xyz), _p(wavelet), _p(rec_offset), _p(rec_xyz),
                              ctypes.c_int(precision), _p(seis), _p(ph), _p(ap))
    if rc != 0:
        raise ValueError("oracle_model: source or receiver outside the model")
    return (seis, ph) if phess else seis


def gradient(g: OGrid, vel, src_xyz, wavelet, rec_offset, rec_xyz, dobs, rho=None,
             snap_every=0, return_seis=False, return_dwav=False, aperture=None):
    """(misfit, dJ/dc [nz][ny][nx]) in FP64; optionally also the modelled
    seismograms and dJ/dw (the wavelet sensitivity)."""
    src_xyz, rec_offset, rec_xyz = _acq(src_xyz, rec_offset, rec_xyz)
    vel, rho, wavelet, dobs = _f64(vel), _f64(rho), _f64(wavelet), _f64(dobs)
    grad = np.zeros((g.nz, g.ny, g.nx))
    seis = np.zeros((int(rec_offset[-1]), g.nt)) if return_seis else None
    dwav = np.zeros(g.nt) if return_dwav else None
    J = ctypes.c_double(0.0)
    ap = _ap(aperture)
    rc = _load().oracle_gradient(ctypes.byref(g), _p(vel), _p(rho), ctypes.c_int(len(src_xyz)),
                                 _p(src_xyz), _p(wavelet), _p(rec_offset), _p(rec_xyz), _p(dobs),
                                 ctypes.c_int(snap_every), ctypes.byref(J), _p(grad), _p(seis),
                                 _p(dwav), _p(ap))
    if rc != 0:
        raise ValueError("oracle_gradient: source or receiver outside the model")
    out = (J.value, grad)
    if return_seis:
        out += (seis,)
    if return_dwav:
        out += (dwav,)
    return out

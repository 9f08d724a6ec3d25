"""Python binding of libmamute (argument marshalling only).

Device arrays are torch CUDA tensors (float32, C-contiguous); geometry
(source and receiver coordinates, receiver offsets, apertures) and the
wavelet are host numpy arrays.  Every computation happens inside the CUDA
library; if the library cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmamute.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mamute.h")

OK, EINVAL, ECFL, ENOMEM, ECUDA, ETIMEOUT, EARCH = 0, -1, -2, -3, -4, -5, -6

_lock = threading.Lock()
_lib = None


class MamuteError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mamute error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("border", ctypes.c_int), ("h", ctypes.c_float), ("dt", ctypes.c_float),
                ("nt", ctypes.c_int), ("ox", ctypes.c_float), ("oy", ctypes.c_float),
                ("oz", ctypes.c_float), ("cerjan", ctypes.c_float), ("free_surface", ctypes.c_int),
                ("xyz_interp", ctypes.c_int), ("pml", ctypes.c_int), ("pml_f0", ctypes.c_float),
                ("pml_r", ctypes.c_float)]


class Opts(ctypes.Structure):
    _fields_ = [("check_mem", ctypes.c_float), ("n_snapshots", ctypes.c_int),
                ("zero_top_planes", ctypes.c_int), ("aperture", ctypes.c_void_p),
                ("phess", ctypes.c_void_p), ("tiles", ctypes.c_int * 6),
                ("smooth_mode", ctypes.c_int), ("smooth_len", ctypes.c_float * 3),
                ("time_interp", ctypes.c_int), ("nt_data", ctypes.c_int),
                ("dt_data", ctypes.c_float), ("time_blocking", ctypes.c_int)]

SMOOTH_NONE, SMOOTH_BESSEL, SMOOTH_LAPLACE = 0, 1, 2
INTERP_NEAREST, INTERP_SINC = 1, 2


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libmamute.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
            lib = ctypes.CDLL(path)
            P, I, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float
            lib.mamute_ctx_create.argtypes = [ctypes.POINTER(P), I, P]
            lib.mamute_ctx_destroy.argtypes = [P]
            lib.mamute_ctx_destroy.restype = None
            lib.mamute_strerror.restype = ctypes.c_char_p
            lib.mamute_strerror.argtypes = [I]
            lib.mamute_last_error.restype = ctypes.c_char_p
            lib.mamute_last_error.argtypes = [P]
            lib.mamute_cfl_limit.restype = D
            common = [P, ctypes.POINTER(Grid), P, P, I, P, P, P, P]
            lib.mamute_model.argtypes = common + [P, P]
            lib.mamute_model_host.argtypes = common + [P, P]
            lib.mamute_gradient.argtypes = common + [P, P, ctypes.POINTER(D), P]
            lib.mamute_gradient_host.argtypes = common + [P, P, ctypes.POINTER(D), P]
            lib.mamute_adjoint.argtypes = common + [P, P, P]
            lib.mamute_gn_diagonal.argtypes = common + [F, P]
            lib.mamute_revolve_plan.argtypes = [I, I, ctypes.POINTER(ctypes.c_longlong),
                                                ctypes.POINTER(I), P]
            lib.mamute_smooth.argtypes = [P, I, I, I, F, I, P, P, P]
            lib.mamute_resample.argtypes = [P, I, I, F, I, F, I, I, P, P]
            _lib = lib
    return _lib


def header_symbols(path: str = HEADER):
    """Function names declared in include/mamute.h."""
    import re
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mamute_\w+)\s*\(", txt)))


def cfl_limit() -> float:
    return float(load().mamute_cfl_limit())


def revolve_plan(nt: int, n_slots: int):
    """(n_forward, actions[n][3]) of the checkpoint schedule (host only)."""
    lib = load()
    nf = ctypes.c_longlong(0)
    na = ctypes.c_int(0)
    rc = lib.mamute_revolve_plan(nt, n_slots, ctypes.byref(nf), ctypes.byref(na), None)
    if rc != OK:
        raise MamuteError(rc, "revolve_plan")
    acts = np.zeros((na.value, 3), dtype=np.int32)
    rc = lib.mamute_revolve_plan(nt, n_slots, ctypes.byref(nf), ctypes.byref(na),
                                 acts.ctypes.data_as(ctypes.c_void_p))
    if rc != OK:
        raise MamuteError(rc, "revolve_plan")
    return int(nf.value), acts


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data_as(ctypes.c_void_p)
    assert t.is_contiguous() and t.dtype.__str__() == "torch.float32", (t.dtype, t.is_contiguous())
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        self._h = ctypes.c_void_p()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        rc = self.lib.mamute_ctx_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(stream))
        if rc != OK:
            raise MamuteError(rc, self.lib.mamute_strerror(rc).decode())
        self.device = device

    def close(self):
        if self._h:
            self.lib.mamute_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise MamuteError(rc, self.lib.mamute_last_error(self._h).decode() or
                              self.lib.mamute_strerror(rc).decode())

    @staticmethod
    def _geom(src_xyz, wavelet, rec_offset, rec_xyz):
        src = np.ascontiguousarray(np.asarray(src_xyz, np.float32).reshape(-1, 3))
        wav = np.ascontiguousarray(wavelet, np.float32)
        off = np.ascontiguousarray(rec_offset, np.int32)
        rec = np.ascontiguousarray(np.asarray(rec_xyz, np.float32).reshape(-1, 3))
        return src, wav, off, rec

    @staticmethod
    def _opts(check_mem=0.8, n_snapshots=0, zero_top_planes=0, aperture=None, phess=None,
              tiles=None, smooth_mode=0, smooth_len=(0.0, 0.0, 0.0), time_interp=0, nt_data=0,
              dt_data=0.0, time_blocking=0):
        ap = None if aperture is None else np.ascontiguousarray(aperture, np.int32)
        o = Opts(check_mem, n_snapshots, zero_top_planes,
                 None if ap is None else ap.ctypes.data, None if phess is None else phess.data_ptr()
                 if not isinstance(phess, np.ndarray) else phess.ctypes.data,
                 (ctypes.c_int * 6)(*(list(tiles) if tiles is not None else [0] * 6)),
                 int(smooth_mode), (ctypes.c_float * 3)(*[float(v) for v in smooth_len]),
                 int(time_interp), int(nt_data), float(dt_data), int(time_blocking))
        return o, ap

    def model(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, seis, **opts):
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        o, keep = self._opts(**opts)
        self._check(self.lib.mamute_model(self._h, ctypes.byref(grid), _ptr(vel), _ptr(rho),
                                          len(src), _ptr(src), _ptr(wav), _ptr(off), _ptr(rec),
                                          ctypes.byref(o), _ptr(seis)))

    def model_host(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, seis, **opts):
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        o, keep = self._opts(**opts)
        self._check(self.lib.mamute_model_host(self._h, ctypes.byref(grid), _ptr(vel), _ptr(rho),
                                               len(src), _ptr(src), _ptr(wav), _ptr(off),
                                               _ptr(rec), ctypes.byref(o), _ptr(seis)))

    def gradient(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, d_obs, grad,
                 **opts) -> float:
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        o, keep = self._opts(**opts)
        J = ctypes.c_double(0.0)
        self._check(self.lib.mamute_gradient(self._h, ctypes.byref(grid), _ptr(vel), _ptr(rho),
                                             len(src), _ptr(src), _ptr(wav), _ptr(off), _ptr(rec),
                                             _ptr(d_obs), ctypes.byref(o), ctypes.byref(J),
                                             _ptr(grad)))
        return J.value

    def gradient_host(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, d_obs,
                      grad, **opts) -> float:
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        o, keep = self._opts(**opts)
        J = ctypes.c_double(0.0)
        self._check(self.lib.mamute_gradient_host(self._h, ctypes.byref(grid), _ptr(vel),
                                                  _ptr(rho), len(src), _ptr(src), _ptr(wav),
                                                  _ptr(off), _ptr(rec), _ptr(d_obs),
                                                  ctypes.byref(o), ctypes.byref(J), _ptr(grad)))
        return J.value

    def adjoint(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, d_res, grad,
                **opts):
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        o, keep = self._opts(**opts)
        self._check(self.lib.mamute_adjoint(self._h, ctypes.byref(grid), _ptr(vel), _ptr(rho),
                                            len(src), _ptr(src), _ptr(wav), _ptr(off), _ptr(rec),
                                            _ptr(d_res), ctypes.byref(o), _ptr(grad)))


    def smooth(self, h: float, mode: int, inp, out, lengths=None):
        """Bessel (mode 1) or Laplace (mode 2) filter of a [nz][ny][nx] tensor."""
        nz, ny, nx = inp.shape
        ln = None if lengths is None else np.ascontiguousarray(lengths, np.float32)
        self._check(self.lib.mamute_smooth(self._h, nx, ny, nz, ctypes.c_float(h), int(mode),
                                           _ptr(ln), _ptr(inp), _ptr(out)))

    def resample(self, x, dt_in: float, nt_out: int, dt_out: float, mode: int, y,
                 adjoint: bool = False, nt_in: int | None = None):
        """Resamples the rows of x [n][nt_in] into y [n][nt_out] (mode 1
        nearest, 2 sinc); adjoint=True applies the transpose (x [n][nt_out]
        -> y [n][nt_in])."""
        n = x.shape[0]
        if adjoint:
            nt_in = y.shape[1]
        else:
            nt_in = x.shape[1]
        self._check(self.lib.mamute_resample(self._h, n, nt_in, ctypes.c_float(dt_in), nt_out,
                                             ctypes.c_float(dt_out), int(mode), int(adjoint),
                                             _ptr(x), _ptr(y)))

    def gn_diagonal(self, grid: Grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, hdiag,
                    band_rel: float = 1e-4):
        src, wav, off, rec = self._geom(src_xyz, wavelet, rec_offset, rec_xyz)
        self._check(self.lib.mamute_gn_diagonal(self._h, ctypes.byref(grid), _ptr(vel), _ptr(rho),
                                                len(src), _ptr(src), _ptr(wav), _ptr(off),
                                                _ptr(rec), ctypes.c_float(band_rel),
                                                _ptr(hdiag)))


def make_grid(nx, ny, nz, border, h, dt, nt, origin=(0.0, 0.0, 0.0), cerjan=0.015,
              free_surface=0, xyz_interp=0, pml=0, pml_f0=0.0, pml_r=0.0) -> Grid:
    return Grid(nx, ny, nz, border, h, dt, nt, origin[0], origin[1], origin[2], cerjan,
                int(free_surface), int(xyz_interp), int(pml), float(pml_f0), float(pml_r))


def grid_of(w, cerjan=0.015, free_surface=0, xyz_interp=0, pml=0, pml_f0=None, pml_r=0.0) -> Grid:
    """Grid of a synthetic workload (see synth.Workload); pml_f0 defaults to
    the workload's peak frequency."""
    f0 = getattr(w, "fpeak", 0.0) if pml_f0 is None else pml_f0
    return make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, cerjan=cerjan,
                     free_surface=free_surface, xyz_interp=xyz_interp, pml=pml, pml_f0=f0,
                     pml_r=pml_r)

"""Gauss-Newton diagonal of the FWI misfit (TEST INFRASTRUCTURE ONLY).

H(x) = sum_s sum_{r in s} sum_m (d d_{s,r}[m] / d c(x))^2, the diagonal of
J^T J for the data of the adjoint-state gradient (Sec. 2.1; Algorithm 3),
with the Born data taken over the full linear-convolution length
m = 0 .. 2 nt - 2 of the nt-step source-side term and the nt-sample impulse
response (reading: "untruncated" window).  With a^n_s(x) = g (lap - m2) u_s^n
and G_{r,x}[k] the response at r of a unit injection at x,
    d d_{s,r}[m] / d A(x) = sum_n G_{r,x}[m - n] a^n_s(x),   dA/dc = 2 c dt^2.

Two independent evaluations:
* ``brute_force``: one forward impulse propagation per cell, explicit
  time-domain convolution, sum of squares;
* ``separable``: one multiplier (adjoint) propagation per receiver gives
  G_{r,x} for all x; Parseval with N_f = 2 nt zero-padded DFT bins gives
  H = (2 c dt^2)^2 (1/N_f) sum_k sum_s sum_{r in s} |G^_r(k)|^2 |a^_s(k)|^2,
  optionally restricted to the bins where the wavelet spectrum exceeds
  band_rel of its peak.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import oracle as O


def _shape(g):
    return (g.nz, g.ny, g.nx)


def forward_terms(g, vel, rho, src_xyz, wavelet, shot):
    a = np.zeros((g.nt,) + _shape(g))
    rc = O._load().oracle_forward_terms(ctypes.byref(g), O._p(O._f64(vel)), O._p(O._f64(rho)),
                                        ctypes.c_int(shot),
                                        O._p(O._f64(np.asarray(src_xyz).reshape(-1, 3))),
                                        O._p(O._f64(wavelet)), O._p(a))
    if rc:
        raise ValueError("source outside the model")
    return a


def cell_response(g, vel, rho, cell, rec_xyz):
    rec = O._f64(np.asarray(rec_xyz).reshape(-1, 3))
    G = np.zeros((len(rec), g.nt))
    rc = O._load().oracle_cell_response(ctypes.byref(g), O._p(O._f64(vel)), O._p(O._f64(rho)),
                                        ctypes.c_int(cell[0]), ctypes.c_int(cell[1]),
                                        ctypes.c_int(cell[2]), ctypes.c_int(len(rec)), O._p(rec),
                                        O._p(G))
    if rc:
        raise ValueError("receiver outside the model")
    return G


def receiver_response(g, vel, rho, rec1):
    G = np.zeros((g.nt,) + _shape(g))
    rc = O._load().oracle_receiver_response(ctypes.byref(g), O._p(O._f64(vel)), O._p(O._f64(rho)),
                                            O._p(O._f64(np.asarray(rec1, np.float64))), O._p(G))
    if rc:
        raise ValueError("receiver outside the model")
    return G


def _dAdc2(g, vel):
    return (2.0 * np.asarray(vel, np.float64) * g.dt**2) ** 2


def brute_force(g, vel, src_xyz, wavelet, rec_offset, rec_xyz, rho=None):
    vel = np.asarray(vel, np.float64)
    src = np.asarray(src_xyz, np.float64).reshape(-1, 3)
    rec = np.asarray(rec_xyz, np.float64).reshape(-1, 3)
    a = [forward_terms(g, vel, rho, src, wavelet, s) for s in range(len(src))]
    H = np.zeros(_shape(g))
    nt = g.nt
    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                G = cell_response(g, vel, rho, (i, j, k), rec)  # [n_rec][nt]
                tot = 0.0
                for s in range(len(src)):
                    aa = a[s][:, k, j, i]
                    for r in range(rec_offset[s], rec_offset[s + 1]):
                        conv = np.zeros(2 * nt - 1)
                        for n in range(nt):
                            conv[n:n + nt] += G[r] * aa[n]
                        tot += np.sum(conv * conv)
                H[k, j, i] = tot
    return H * _dAdc2(g, vel)


def band_bins(wavelet, nt, band_rel):
    nf = 2 * nt
    spec = np.abs(np.fft.rfft(np.asarray(wavelet, np.float64), nf))
    if band_rel is None or band_rel <= 0:
        return np.arange(nf // 2 + 1)
    return np.nonzero(spec >= band_rel * spec.max())[0]


def separable(g, vel, src_xyz, wavelet, rec_offset, rec_xyz, rho=None, band_rel=None):
    vel = np.asarray(vel, np.float64)
    src = np.asarray(src_xyz, np.float64).reshape(-1, 3)
    rec = np.asarray(rec_xyz, np.float64).reshape(-1, 3)
    nt, nf = g.nt, 2 * g.nt
    bins = band_bins(wavelet, nt, band_rel)
    w = np.where((bins == 0) | (bins == nf // 2), 1.0, 2.0)  # rfft weights for the full sum
    Ahat = [np.fft.rfft(forward_terms(g, vel, rho, src, wavelet, s), nf, axis=0)[bins]
            for s in range(len(src))]
    H = np.zeros(_shape(g))
    Ghat = {}
    for r in range(len(rec)):
        Ghat[r] = np.fft.rfft(receiver_response(g, vel, rho, rec[r]), nf, axis=0)[bins]
    for s in range(len(src)):
        S = np.abs(Ahat[s]) ** 2
        for r in range(rec_offset[s], rec_offset[s + 1]):
            H += np.tensordot(w, np.abs(Ghat[r]) ** 2 * S, axes=(0, 0))
    return H * _dAdc2(g, vel) / nf

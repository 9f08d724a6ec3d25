"""Gradient smoothing and seismic-data time resampling (TEST INFRASTRUCTURE ONLY).

Plain, slow restatements used only by the tests, the smoke check and the
benchmark's CPU baseline; the product library never imports this module.

Gradient preconditioning (Sec. 2, FWI: "no filter, Bessel filter, or Laplace
filter" with lengths bessel_filter_l{x,y,z}, default two grid spacings;
Algorithm 3: GradientPreconditioning, then ZeroesNearSurface).  Reading: the
Bessel filter (after the smoothing operator the paper cites) solves
    (I - lx^2 Dxx - ly^2 Dyy - lz^2 Dzz) u = g,
whose continuous kernel in 3-D is exp(-r/l) / (4 pi l^2 r), a modified
spherical Bessel function; the Laplace filter is the separable product
    u = (I - lx^2 Dxx)^-1 (I - ly^2 Dyy)^-1 (I - lz^2 Dzz)^-1 g,
whose 1-D factors have the Laplace-distribution kernel exp(-|x|/l) / (2 l).
D_aa is the 3-point second difference on the model grid with reflecting
ends (the value beyond the last cell repeats it), so constants pass
unchanged.  Both are written here as the linear systems themselves, solved
with library solvers.

Time resampling (Sec. 2: "time interpolation via the nearest neighbour
algorithm or sinc function"; Table 1 Interpolate).  Sample n of a trace
sits at time n dt_in, output sample m at time m dt_out.  Nearest: y[m] =
x[floor(m dt_out / dt_in + 1/2)] (zero past the trace).  Sinc (reading): a
Hann-tapered band-limited kernel of half-width W = 8 samples of the coarser
step D = max(dt_in, dt_out):
    y[m] = sum_n x[n] (dt_in / D) sinc((t_m - n dt_in) / D) hann((t_m - n dt_in) / (W D)),
hann(u) = (1 + cos(pi u)) / 2 for |u| < 1, else 0; for dt_out <= dt_in this
is interpolation, for dt_out > dt_in it low-passes below the output Nyquist
frequency before decimating.  The adjoint (used to bring data residuals back
to the modelling time axis) is the transpose of the same matrix.
"""
from __future__ import annotations

import numpy as np

SINC_HALF_WIDTH = 8


# ------------------------------------------------------------ smoothing
def second_difference(n: int) -> np.ndarray:
    """n x n matrix of u[i-1] - 2 u[i] + u[i+1] with reflecting ends."""
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = -2.0
        D[i, max(i - 1, 0)] += 1.0
        D[i, min(i + 1, n - 1)] += 1.0
    return D


def _axis_operator(n: int, length: float, h: float) -> np.ndarray:
    return np.eye(n) - (length / h) ** 2 * second_difference(n)


def laplace_filter(g, h, lengths):
    """Separable filter: (I - l^2 D)^-1 along x, y and z in turn (g is [z][y][x])."""
    u = np.asarray(g, np.float64)
    lx, ly, lz = lengths
    for axis, length in ((2, lx), (1, ly), (0, lz)):
        T = _axis_operator(u.shape[axis], length, h)
        u = np.moveaxis(np.linalg.solve(T, np.moveaxis(u, axis, 0).reshape(u.shape[axis], -1))
                        .reshape(np.moveaxis(u, axis, 0).shape), 0, axis)
    return u


def bessel_filter(g, h, lengths):
    """Non-separable filter: (I - lx^2 Dxx - ly^2 Dyy - lz^2 Dzz) u = g, one
    sparse direct solve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    g = np.asarray(g, np.float64)
    nz, ny, nx = g.shape
    lx, ly, lz = lengths
    Dx = sp.csr_matrix(second_difference(nx))
    Dy = sp.csr_matrix(second_difference(ny))
    Dz = sp.csr_matrix(second_difference(nz))
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    # C-order [z][y][x]: x is the fastest index, so it is the last Kronecker factor
    L = ((lx / h) ** 2 * sp.kron(sp.kron(Iz, Iy), Dx) + (ly / h) ** 2 * sp.kron(sp.kron(Iz, Dy), Ix)
         + (lz / h) ** 2 * sp.kron(sp.kron(Dz, Iy), Ix))
    A = sp.identity(nx * ny * nz) - L
    return spl.spsolve(A.tocsc(), g.ravel()).reshape(g.shape)


def smooth(g, h, mode, lengths=None):
    """mode 0: none, 1: Bessel, 2: Laplace; lengths default to 2 h each."""
    if lengths is None:
        lengths = (2 * h, 2 * h, 2 * h)
    if mode == 0:
        return np.asarray(g, np.float64).copy()
    if mode == 1:
        return bessel_filter(g, h, lengths)
    if mode == 2:
        return laplace_filter(g, h, lengths)
    raise ValueError("mode must be 0, 1 or 2")


# ------------------------------------------------------------ resampling
def resample_matrix(nt_in: int, dt_in: float, nt_out: int, dt_out: float, mode: str,
                    half_width: int = SINC_HALF_WIDTH) -> np.ndarray:
    """The [nt_out][nt_in] matrix of the resampling (see the module text)."""
    K = np.zeros((nt_out, nt_in))
    if mode == "nearest":
        for m in range(nt_out):
            n = int(np.floor(m * dt_out / dt_in + 0.5))
            if 0 <= n < nt_in:
                K[m, n] = 1.0
        return K
    if mode != "sinc":
        raise ValueError("mode must be 'nearest' or 'sinc'")
    D = max(dt_in, dt_out)
    for m in range(nt_out):
        for n in range(nt_in):
            u = (m * dt_out - n * dt_in) / D
            if abs(u) < half_width:
                K[m, n] = dt_in / D * np.sinc(u) * 0.5 * (1.0 + np.cos(np.pi * u / half_width))
    return K


def resample(x, dt_in, nt_out, dt_out, mode, adjoint=False, nt_in=None):
    """Resamples the rows of x ([n][nt_in] -> [n][nt_out]); with adjoint=True
    applies the transpose ([n][nt_out] -> [n][nt_in], nt_in given)."""
    x = np.asarray(x, np.float64)
    if adjoint:
        K = resample_matrix(nt_in, dt_in, x.shape[-1], dt_out, mode)
        return x @ K
    K = resample_matrix(x.shape[-1], dt_in, nt_out, dt_out, mode)
    return x @ K.T

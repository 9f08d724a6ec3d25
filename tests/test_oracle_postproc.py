"""Pins of the oracle's gradient smoothing filters and data resampling.

The filters are pinned by closed forms: products of DCT-II cosines are their
eigenvectors (reflecting ends) with eigenvalues written out here, constants
pass unchanged, the 1-D kernel of (1 - l^2 D)^-1 is a geometric sequence whose
ratio solves a quadratic, and the 3-D Bessel kernel approaches
exp(-r/l) / (4 pi l^2 r) for lengths of several cells.  The resampling is
pinned by the identity at equal steps, exact index picking, band-limited
reconstruction of sinusoids, and the attenuation of frequencies above the
output Nyquist frequency when decimating.
"""
import numpy as np
import pytest

from oracle import postproc


def _dct_mode(shape, k):
    nz, ny, nx = shape
    kz, ky, kx = k
    cz = np.cos(np.pi * kz * (np.arange(nz) + 0.5) / nz)
    cy = np.cos(np.pi * ky * (np.arange(ny) + 0.5) / ny)
    cx = np.cos(np.pi * kx * (np.arange(nx) + 0.5) / nx)
    return cz[:, None, None] * cy[None, :, None] * cx[None, None, :]


@pytest.mark.parametrize("k", [(0, 0, 0), (1, 0, 3), (2, 5, 1), (6, 6, 8)])
def test_filters_act_on_dct_modes_by_closed_form_eigenvalues(k):
    shape, h = (7, 9, 11), 10.0
    lengths = (20.0, 13.0, 31.0)  # lx, ly, lz
    g = _dct_mode(shape, k)
    lam = [4 * (L / h) ** 2 * np.sin(np.pi * kk / (2 * n)) ** 2
           for L, kk, n in zip((lengths[2], lengths[1], lengths[0]), k, shape)]
    bes = postproc.smooth(g, h, 1, lengths)
    lap = postproc.smooth(g, h, 2, lengths)
    np.testing.assert_allclose(bes, g / (1 + sum(lam)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(lap, g / np.prod([1 + x for x in lam]), rtol=0, atol=1e-12)


def test_filters_keep_constants_and_are_symmetric():
    rng = np.random.default_rng(0)
    shape, h = (6, 8, 5), 12.5
    c = np.full(shape, 3.25)
    for mode in (1, 2):
        np.testing.assert_allclose(postproc.smooth(c, h, mode), c, rtol=1e-13)
        a, b = rng.standard_normal(shape), rng.standard_normal(shape)
        lhs = np.sum(postproc.smooth(a, h, mode) * b)
        rhs = np.sum(a * postproc.smooth(b, h, mode))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    np.testing.assert_array_equal(postproc.smooth(c, h, 0), c)


def test_one_dimensional_kernel_is_geometric():
    """(1 - a D) u = delta on a long line: u_k = u_0 r^|k| with
    a r^2 - (1 + 2a) r + a = 0 and u_0 = 1 / (1 + 2a - 2a r)."""
    n, h, L = 201, 1.0, 3.0
    a = (L / h) ** 2
    g = np.zeros((1, 1, n))
    g[0, 0, n // 2] = 1.0
    u = postproc.smooth(g, h, 2, (L, 1.0, 1.0))[0, 0]
    r = ((1 + 2 * a) - np.sqrt((1 + 2 * a) ** 2 - 4 * a * a)) / (2 * a)
    u0 = 1.0 / (1 + 2 * a - 2 * a * r)
    k = np.arange(-40, 41)
    np.testing.assert_allclose(u[n // 2 + k], u0 * r ** np.abs(k), rtol=1e-10)
    # and the continuous Laplace-distribution kernel for a length of several cells
    assert abs(u0 - h / (2 * L)) < 0.1 * h / (2 * L)


def test_bessel_kernel_approaches_its_continuous_form():
    n, h, L = 33, 1.0, 3.0
    g = np.zeros((n, n, n))
    c = n // 2
    g[c, c, c] = 1.0 / h**3
    u = postproc.smooth(g, h, 1, (L, L, L))
    for r in (4, 6, 8):
        exact = np.exp(-r / L) / (4 * np.pi * L * L * r)
        assert abs(u[c, c, c + r] - exact) < 0.06 * exact, (r, u[c, c, c + r], exact)


def test_resample_identity_and_nearest():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 50))
    for mode in ("nearest", "sinc"):
        np.testing.assert_allclose(postproc.resample(x, 1e-3, 50, 1e-3, mode), x, rtol=0,
                                   atol=1e-13)
    y = postproc.resample(x, 1e-3, 25, 2e-3, "nearest")
    np.testing.assert_array_equal(y, x[:, ::2])
    # half-way samples round up (floor(t/dt + 1/2)); beyond the trace: zero
    y = postproc.resample(x, 2e-3, 101, 1e-3, "nearest")
    np.testing.assert_array_equal(y[:, 1], x[:, 1])
    np.testing.assert_array_equal(y[:, 99:], 0.0)


def test_sinc_reconstructs_band_limited_signals():
    dt, nt = 4e-3, 160
    t = np.arange(nt) * dt
    f = [7.0, 23.0, 41.0]  # below 0.4 of the 125 Hz Nyquist frequency
    sig = lambda tt: sum(np.sin(2 * np.pi * fi * tt + i) for i, fi in enumerate(f))
    x = sig(t)[None, :]
    dt_out = 1e-3
    y = postproc.resample(x, dt, 600, dt_out, "sinc")[0]
    to = np.arange(600) * dt_out
    inner = (to > 10 * dt) & (to < (nt - 10) * dt)
    err = np.abs(y[inner] - sig(to[inner])).max()
    assert err < 1e-2, err


def test_sinc_decimation_removes_frequencies_above_the_output_nyquist():
    dt_in, nt = 1e-3, 2000
    t = np.arange(nt) * dt_in
    dt_out = 4e-3  # output Nyquist 125 Hz
    to = np.arange(nt // 4) * dt_out
    for f, passes in ((40.0, True), (200.0, False)):
        x = np.sin(2 * np.pi * f * t)[None, :]
        y = postproc.resample(x, dt_in, nt // 4, dt_out, "sinc")[0]
        if passes:  # the passband goes through unchanged: the sinusoid at the output times
            err = np.abs(y[50:-50] - np.sin(2 * np.pi * f * to[50:-50])).max()
            assert err < 0.05, (f, err)
        else:
            amp = np.abs(y[50:-50]).max()
            assert amp < 0.05, (f, amp)


def test_resample_adjoint_is_the_transpose():
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((2, 70)), rng.standard_normal((2, 31))
    for mode in ("nearest", "sinc"):
        Kx = postproc.resample(x, 1e-3, 31, 2.3e-3, mode)
        KTy = postproc.resample(y, 1e-3, None, 2.3e-3, mode, adjoint=True, nt_in=70)
        assert abs(np.sum(Kx * y) - np.sum(x * KTy)) < 1e-12 * np.abs(Kx * y).sum()

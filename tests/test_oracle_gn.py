"""Pins of the Gauss-Newton diagonal oracle: the brute-force definition (one
forward impulse propagation per cell, time-domain convolution) and the
separable form (one multiplier propagation per receiver, Parseval over
2 nt DFT bins) agree to rounding; the band limit used for labels costs
little for a Ricker source."""
import numpy as np

from oracle import gn
from paper_2502_12350_gb300 import synth


def _case(density, nt, seed):
    return synth.small_case(seed=seed, nx=6, ny=5, nz=5, border=4, nt=nt, density=density,
                            n_src=2, n_rec=3, fpeak=40.0)


def test_brute_force_equals_separable(oracle):
    for density in (False, True):
        w = _case(density, 40, 51)
        g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
        Hb = gn.brute_force(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
        Hs = gn.separable(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
        assert Hb.min() > 0
        np.testing.assert_allclose(Hs, Hb, rtol=1e-10)


def test_band_limit_error_small(oracle):
    w = _case(False, 120, 52)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    Hs = gn.separable(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz)
    Hl = gn.separable(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, band_rel=1e-4)
    assert len(gn.band_bins(w.wavelet, w.nt, 1e-4)) < w.nt // 2
    assert np.abs(Hl - Hs).max() / Hs.max() < 1e-4


def test_gn_diagonal_scales_with_source_energy(oracle):
    """H is quadratic in the wavelet amplitude (a linear source term)."""
    w = _case(True, 40, 53)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    H1 = gn.separable(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    H3 = gn.separable(g, w.vel, w.src_xyz, 3.0 * w.wavelet.astype(np.float64), w.rec_offset,
                      w.rec_xyz, rho=w.rho)
    np.testing.assert_allclose(H3, 9.0 * H1, rtol=1e-12)

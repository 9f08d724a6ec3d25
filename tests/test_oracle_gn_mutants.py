"""The Gauss-Newton-diagonal pins fail for plausible mistakes in the
oracle: each mutant replaces one function of oracle.gn (on the CPU, for the
duration of one test) and the named pin must fail, while the unmodified
module passes it."""
import numpy as np
import pytest

from oracle import gn

import test_oracle_gn as gn_pins
import test_oracle_pins as pins


def _dAdc2_without_2(g, vel):
    return (np.asarray(vel, np.float64) * g.dt**2) ** 2


def _separable_unit_weights(g, vel, src_xyz, wavelet, rec_offset, rec_xyz, rho=None,
                            band_rel=None):
    """The separable form with every rfft bin counted once (the interior bins
    stand for two bins of the full spectrum)."""
    vel = np.asarray(vel, np.float64)
    src = np.asarray(src_xyz, np.float64).reshape(-1, 3)
    rec = np.asarray(rec_xyz, np.float64).reshape(-1, 3)
    nt, nf = g.nt, 2 * g.nt
    bins = gn.band_bins(wavelet, nt, band_rel)
    w = np.ones(len(bins))
    Ahat = [np.fft.rfft(gn.forward_terms(g, vel, rho, src, wavelet, s), nf, axis=0)[bins]
            for s in range(len(src))]
    H = np.zeros(gn._shape(g))
    for s in range(len(src)):
        S = np.abs(Ahat[s]) ** 2
        for r in range(rec_offset[s], rec_offset[s + 1]):
            Gh = np.fft.rfft(gn.receiver_response(g, vel, rho, rec[r]), nf, axis=0)[bins]
            H += np.tensordot(w, np.abs(Gh) ** 2 * S, axes=(0, 0))
    return H * gn._dAdc2(g, vel) / nf


def test_chain_rule_factor_is_pinned(oracle, monkeypatch):
    pins.test_gn_jacobian_column_matches_finite_differences(oracle, False)
    monkeypatch.setattr(gn, "_dAdc2", _dAdc2_without_2)
    with pytest.raises(AssertionError):
        pins.test_gn_jacobian_column_matches_finite_differences(oracle, False)


def test_parseval_weights_are_pinned(oracle, monkeypatch):
    gn_pins.test_brute_force_equals_separable(oracle)
    monkeypatch.setattr(gn, "separable", _separable_unit_weights)
    with pytest.raises(AssertionError):
        gn_pins.test_brute_force_equals_separable(oracle)

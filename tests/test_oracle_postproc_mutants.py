"""The smoothing and resampling pins fail for plausible mistakes in the
oracle: each mutant replaces one function of oracle.postproc (on the CPU,
for the duration of one test) and the named pin must fail, while the
unmodified module passes every one of them."""
import numpy as np
import pytest

from oracle import postproc as P

import test_oracle_postproc as pins

_resample_matrix = P.resample_matrix
_laplace_filter = P.laplace_filter


def _dirichlet_ends(n):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = -2.0
        if i > 0:
            D[i, i - 1] = 1.0
        if i < n - 1:
            D[i, i + 1] = 1.0
    return D


def _length_not_squared(n, length, h):
    return np.eye(n) - (length / h) * P.second_difference(n)


def _laplace_without_z(g, h, lengths):
    return _laplace_filter(g, h, (lengths[0], lengths[1], 0.0))


def _resampling(kind):
    def resample_matrix(nt_in, dt_in, nt_out, dt_out, mode, half_width=P.SINC_HALF_WIDTH):
        if mode == "nearest" and kind == "floor for nearest":
            K = np.zeros((nt_out, nt_in))
            for m in range(nt_out):
                n = int(np.floor(m * dt_out / dt_in))
                if 0 <= n < nt_in:
                    K[m, n] = 1.0
            return K
        if mode != "sinc":
            return _resample_matrix(nt_in, dt_in, nt_out, dt_out, mode, half_width)
        K = np.zeros((nt_out, nt_in))
        D = max(dt_in, dt_out)
        for m in range(nt_out):
            for n in range(nt_in):
                u = (m * dt_out - n * dt_in) / D
                if abs(u) < half_width:
                    amp = 1.0 if kind == "sinc without dt_in / D" else dt_in / D
                    win = 1.0 if kind == "sinc without window" else \
                        0.5 * (1.0 + np.cos(np.pi * u / half_width))
                    K[m, n] = amp * np.sinc(u) * win
        return K
    return resample_matrix


# name: (function replaced, replacement, pin that must fail, its parameters)
MUTANTS = {
    "reflecting ends dropped": ("second_difference", _dirichlet_ends,
                                pins.test_filters_keep_constants_and_are_symmetric, ()),
    "l / h not squared": ("_axis_operator", _length_not_squared,
                          pins.test_one_dimensional_kernel_is_geometric, ()),
    "Laplace filter without its z pass": (
        "laplace_filter", _laplace_without_z,
        pins.test_filters_act_on_dct_modes_by_closed_form_eigenvalues, ((1, 0, 3),)),
    "floor for nearest": ("resample_matrix", _resampling("floor for nearest"),
                          pins.test_resample_identity_and_nearest, ()),
    "sinc without dt_in / D": (
        "resample_matrix", _resampling("sinc without dt_in / D"),
        pins.test_sinc_decimation_removes_frequencies_above_the_output_nyquist, ()),
    "sinc without window": ("resample_matrix", _resampling("sinc without window"),
                            pins.test_sinc_reconstructs_band_limited_signals, ()),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_fails_its_pin(monkeypatch, name):
    attr, fn, pin, args = MUTANTS[name]
    pin(*args)  # the unmodified oracle passes it
    monkeypatch.setattr(P, attr, fn)
    with pytest.raises(AssertionError):
        pin(*args)

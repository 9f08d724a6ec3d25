"""The CPML coefficient pins fail for plausible mistakes in the oracle's
layer profiles: each mutant below replaces oracle.cpml.profiles (on the CPU,
for the duration of one test) and at least one pin must fail for it, while
the unmodified profiles pass both."""
import numpy as np
import pytest

from oracle import cpml

import test_oracle_cpml as pins

PINS = (pins.test_layer_reaches_the_nominal_reflection,
        pins.test_recursion_is_the_convolution_with_the_layer_kernel)


def _mutant(kind):
    def profiles(N, border, h, dt, vmax, f0, R=1e-3, low_face=True):
        L = border * h
        k = 2.0 if kind == "factor 2 for 3" else 3.0
        lnR = np.log10(R) if kind == "log10 for ln" else np.log(R)
        d0 = -k * vmax * lnR / (2.0 * L)
        dist = np.zeros(N)
        for i in range(N):
            if i < border:
                dist[i] = border - i if low_face else 0
            elif i > N - 1 - border:
                dist[i] = i - (N - 1 - border)
        r = dist / max(border, 1)
        shape = r if kind == "linear profile" else r * r
        d = np.where(dist > 0, d0 * shape, 0.0)
        alpha = np.where(dist > 0, np.pi * f0 * (1.0 - r), 0.0)
        b = np.exp(-(d if kind == "b without alpha" else d + alpha) * dt)
        c = np.where(d + alpha > 0, d * (b - 1.0) / np.where(d + alpha > 0, d + alpha, 1.0), 0.0)
        if kind == "sign of c":
            c = -c
        return b, c
    return profiles


def _failures(monkeypatch, kind):
    monkeypatch.setattr(cpml, "profiles", _mutant(kind))
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    return failed


def test_unmodified_profiles_pass(monkeypatch):
    assert _failures(monkeypatch, "none") == 0


@pytest.mark.parametrize("kind", ["factor 2 for 3", "log10 for ln", "linear profile",
                                  "b without alpha", "sign of c"])
def test_mutant_fails_a_pin(monkeypatch, kind):
    assert _failures(monkeypatch, kind) >= 1

"""The conv3d oracle's pins fail for plausible mistakes: each mutant
replaces one function of oracle.conv (on the CPU, for the duration of one
test) and the named pin must fail, while the unmodified module passes it."""
import numpy as np
import pytest

from oracle import conv

import test_oracle_conv as pins


def _forward_flipped(x, w, b=None):
    """A convolution (flipped taps) instead of the cross-correlation."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    D, H, W = x.shape[1:]
    xp = conv._pad(x)
    y = np.zeros((w.shape[0], D, H, W))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, 2 - dz:2 - dz + D, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W]
                y += np.tensordot(w[:, :, dz, dy, dx], patch, axes=(1, 0))
    if b is not None:
        y += np.asarray(b, np.float64)[:, None, None, None]
    return y


def _backward_input_unflipped(gy, w):
    gy = np.asarray(gy, np.float64)
    w = np.asarray(w, np.float64)
    D, H, W = gy.shape[1:]
    gp = conv._pad(gy)
    gx = np.zeros((w.shape[1], D, H, W))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = gp[:, dz:dz + D, dy:dy + H, dx:dx + W]
                gx += np.tensordot(w[:, :, dz, dy, dx], patch, axes=(0, 0))
    return gx


def _backward_weight_shifted(x, gy):
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    D, H, W = x.shape[1:]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (2, 0)))  # x window one cell off
    gw = np.zeros((gy.shape[0], x.shape[0], 3, 3, 3))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + D, dy:dy + H, dx:dx + W]
                gw[:, :, dz, dy, dx] = np.tensordot(gy, patch, axes=([1, 2, 3], [1, 2, 3]))
    return gw, gy.sum(axis=(1, 2, 3))


def _bf16_truncate(a):
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32) & np.uint32(0xFFFF0000)
    return u.view(np.float32).astype(np.float64)


def _bf16_ties_away(a):
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x8000) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


MUTANTS = {
    "convolution for cross-correlation": ("forward", _forward_flipped,
                                          pins.test_forward_matches_torch_conv3d),
    "input gradient not flipped": ("backward_input", _backward_input_unflipped,
                                   pins.test_adjoint_identities),
    "weight gradient one cell off": ("backward_weight", _backward_weight_shifted,
                                     pins.test_adjoint_identities),
    "BF16 by truncation": ("bf16_round", _bf16_truncate, pins.test_bf16_rounding_rule),
    "BF16 ties away from zero": ("bf16_round", _bf16_ties_away, pins.test_bf16_rounding_rule),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_fails_its_pin(monkeypatch, name):
    attr, fn, pin = MUTANTS[name]
    pin()  # the unmodified oracle passes it
    monkeypatch.setattr(conv, attr, fn)
    with pytest.raises(AssertionError):
        pin()

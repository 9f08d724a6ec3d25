"""3x3x3 'same' convolution, FP64 (TEST INFRASTRUCTURE ONLY).

The learned preconditioner's network (4 layers, 3^3 kernels, 16 channels,
ReLU) runs on BF16 inputs with FP32 accumulation; the oracle rounds its
inputs to BF16 (round to nearest even) and then computes in FP64 by the
textbook sums:

  forward      y[o, z, y, x] = b[o] + sum_{i, dz, dy, dx} w[o, i, dz, dy, dx]
                                 * x[i, z+dz-1, y+dy-1, x+dx-1]      (zero outside)
  d input      gx[i, p] = sum_{o, d} w[o, i, d] gy[o, p - d + 1]
  d weight     gw[o, i, d] = sum_p gy[o, p] x[i, p + d - 1]
  d bias       gb[o] = sum_p gy[o, p]

Layout [C][D][H][W] (channels first) for readability; the CUDA path uses
channels last.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest BF16 value (ties to even), as FP64."""
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(x)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))


def forward(x, w, b=None):
    """x [Ci][D][H][W], w [Co][Ci][3][3][3], b [Co] -> y [Co][D][H][W] (FP64)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    Co, Ci = w.shape[:2]
    D, H, W = x.shape[1:]
    xp = _pad(x)
    y = np.zeros((Co, D, H, W))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + D, dy:dy + H, dx:dx + W]      # [Ci][D][H][W]
                y += np.tensordot(w[:, :, dz, dy, dx], patch, axes=(1, 0))
    if b is not None:
        y += np.asarray(b, np.float64)[:, None, None, None]
    return y


def backward_input(gy, w):
    """gy [Co][D][H][W], w [Co][Ci][3][3][3] -> gx [Ci][D][H][W]."""
    gy = np.asarray(gy, np.float64)
    w = np.asarray(w, np.float64)
    D, H, W = gy.shape[1:]
    gp = _pad(gy)
    gx = np.zeros((w.shape[1], D, H, W))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                # gx[i, p] += w[o, i, d] gy[o, p - d + 1]
                patch = gp[:, 2 - dz:2 - dz + D, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W]
                gx += np.tensordot(w[:, :, dz, dy, dx], patch, axes=(0, 0))
    return gx


def backward_weight(x, gy):
    """x [Ci][D][H][W], gy [Co][D][H][W] -> (gw [Co][Ci][3][3][3], gb [Co])."""
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    D, H, W = x.shape[1:]
    xp = _pad(x)
    gw = np.zeros((gy.shape[0], x.shape[0], 3, 3, 3))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + D, dy:dy + H, dx:dx + W]
                gw[:, :, dz, dy, dx] = np.tensordot(gy, patch, axes=([1, 2, 3], [1, 2, 3]))
    return gw, gy.sum(axis=(1, 2, 3))


class Net:
    """The preconditioner network in FP64 on BF16-rounded inputs and weights:
    conv(2->16) ReLU conv(16->16) ReLU conv(16->16) ReLU conv(16->1)."""

    def __init__(self, weights, biases, round_activations=True):
        self.w = [bf16_round(w) for w in weights]
        self.b = [np.asarray(b, np.float64) for b in biases]
        # The network stores activations in BF16; the gradients treat that
        # rounding as the identity.  round_activations=False gives the
        # unrounded network whose exact gradient those formulas are.
        self.rnd = bf16_round if round_activations else (lambda a: np.asarray(a, np.float64))

    def forward(self, x):
        acts = [self.rnd(x)]
        h = acts[0]
        pre = []
        for l in range(4):
            z = forward(h, self.w[l], self.b[l])
            pre.append(z)
            if l < 3:
                h = self.rnd(np.maximum(z, 0.0))
                acts.append(h)
        return z, acts, pre

    def loss_and_grads(self, x, target, mask=None):
        """Mean squared error over the voxels (mask selects them) and its
        gradients with respect to the weights and biases."""
        out, acts, pre = self.forward(x)
        m = np.ones_like(out[0]) if mask is None else np.asarray(mask, np.float64)
        n = m.sum()
        r = (out[0] - target) * m
        loss = np.sum(r * r) / n
        g = (2.0 / n) * r[None]
        gws, gbs = [None] * 4, [None] * 4
        for l in range(3, -1, -1):
            gws[l], gbs[l] = backward_weight(acts[l], g)
            if l > 0:
                g = backward_input(g, self.w[l]) * (pre[l - 1] > 0)
        return loss, gws, gbs

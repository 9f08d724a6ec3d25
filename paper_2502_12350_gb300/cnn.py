"""The learned Gauss-Newton-diagonal preconditioner network (driver).

A 4-layer 3x3x3 'same' CNN, conv(2->16) ReLU conv(16->16) ReLU
conv(16->16) ReLU conv(16->1), maps (normalised velocity, log
pseudo-Hessian) to log(H / P) - offset, H the Gauss-Newton diagonal and
P the pseudo-Hessian.  Every
convolution, gradient, loss and optimizer update runs in libmamute's
kernels (BF16 products, FP32 accumulation and masters); this module only
holds the device buffers (torch tensors as memory) and sequences the calls.
Channel counts below 16 are zero-padded to 16 throughout.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import mamute

C = 16
TAPS = 27
LAYERS = 4
CHANNELS = [2, 16, 16, 16, 1]


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _bind(lib):
    P, I, F, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_longlong
    lib.mamute_conv3d.argtypes = [P, I, I, I, P, P, P, I, P, P, P]
    lib.mamute_conv3d_wgrad.argtypes = [P, I, I, I, P, P, P, P]
    lib.mamute_conv3d_pack.argtypes = [P, P, P, P]
    lib.mamute_mse_loss.argtypes = [P, LL, P, P, P, D, ctypes.POINTER(D), P]
    lib.mamute_adam.argtypes = [P, I, P, P, P, P, F, F, F, F, I]
    lib.mamute_nn_features.argtypes = [P, LL, P, P, P, F, F, F, P, P, ctypes.POINTER(F)]
    return lib


def init_weights(seed: int = 0):
    """He-initialised masters [27][16 out][16 in] per layer (padding zero)."""
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for l in range(LAYERS):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        w = np.zeros((TAPS, C, C), np.float32)
        w[:, :co, :ci] = rng.standard_normal((TAPS, co, ci)) * np.sqrt(2.0 / (TAPS * ci))
        if l == LAYERS - 1:
            w *= 0.1
        ws.append(w)
        bs.append(np.zeros(C, np.float32))
    return ws, bs


def to_oracle_layout(w):
    """[27][o][i] -> [o][i][3][3][3] (taps in (dz, dy, dx) order)."""
    return np.transpose(np.asarray(w).reshape(3, 3, 3, C, C), (3, 4, 0, 1, 2))


class Net:
    def __init__(self, ctx: mamute.Context, seed: int = 0, weights=None):
        self.ctx = ctx
        self.lib = _bind(ctx.lib)
        self.dev = torch.device("cuda", ctx.device)
        ws, bs = weights if weights is not None else init_weights(seed)
        self.w = [torch.from_numpy(np.ascontiguousarray(w)).to(self.dev) for w in ws]
        self.b = [torch.from_numpy(np.ascontiguousarray(b)).to(self.dev) for b in bs]
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.gw = [torch.zeros_like(w) for w in self.w]
        self.gb = [torch.zeros_like(b) for b in self.b]
        self.wf = [torch.zeros((TAPS, C, C), dtype=torch.int16, device=self.dev) for _ in ws]
        self.wb = [torch.zeros((TAPS, C, C), dtype=torch.int16, device=self.dev) for _ in ws]
        self.step = 0
        self.offset = 0.0  # added to the output: prediction of log(H / P)
        self._shape = None
        self.pack()

    def _check(self, rc):
        self.ctx._check(rc)

    def pack(self):
        for l in range(LAYERS):
            self._check(self.lib.mamute_conv3d_pack(self.ctx._h, _p(self.w[l]), _p(self.wf[l]),
                                                    _p(self.wb[l])))

    def _buffers(self, shape):
        if self._shape != shape:
            D, H, W = shape
            self.acts = [torch.zeros((D, H, W, C), dtype=torch.int16, device=self.dev)
                         for _ in range(LAYERS)]
            self.out = torch.zeros((D, H, W, C), dtype=torch.float32, device=self.dev)
            self.g16 = [torch.zeros((D, H, W, C), dtype=torch.int16, device=self.dev)
                        for _ in range(2)]
            self._shape = shape

    def features(self, vel, phess, hdiag=None, v_ref=3000.0, v_scale=1000.0, log_clip=20.0):
        """(x16 [D][H][W][16] BF16, target or None, Pmax) for one model."""
        D, H, W = vel.shape
        x16 = torch.zeros((D, H, W, C), dtype=torch.int16, device=self.dev)
        tgt = torch.zeros((D, H, W), dtype=torch.float32, device=self.dev) if hdiag is not None else None
        pmax = ctypes.c_float(0.0)
        self._check(self.lib.mamute_nn_features(self.ctx._h, vel.numel(), _p(vel), _p(phess),
                                                _p(hdiag), v_ref, v_scale, log_clip, _p(x16),
                                                _p(tgt), ctypes.byref(pmax)))
        return x16, tgt, pmax.value

    def forward(self, x16):
        """Network output (channel 0 of an FP32 [D][H][W][16] tensor)."""
        D, H, W = x16.shape[:3]
        self._buffers((D, H, W))
        self.acts[0].copy_(x16)
        h = self.acts[0]
        for l in range(LAYERS):
            last = l == LAYERS - 1
            self._check(self.lib.mamute_conv3d(
                self.ctx._h, D, H, W, _p(h), _p(self.wf[l]), _p(self.b[l]), 0 if last else 1, None,
                _p(self.out) if last else None, None if last else _p(self.acts[l + 1])))
            if not last:
                h = self.acts[l + 1]
        return self.out[..., 0]

    def loss_and_grads(self, x16, target, mask=None, n_mask=None):
        """Forward, masked MSE and backward; fills self.gw / self.gb."""
        D, H, W = x16.shape[:3]
        self.forward(x16)
        n = D * H * W
        n_mask = float(n if mask is None else (n_mask if n_mask is not None else mask.sum().item()))
        loss = ctypes.c_double(0.0)
        g = self.g16[0]
        self._check(self.lib.mamute_mse_loss(self.ctx._h, n, _p(self.out), _p(target), _p(mask),
                                             n_mask, ctypes.byref(loss), _p(g)))
        for l in range(LAYERS - 1, -1, -1):
            self._check(self.lib.mamute_conv3d_wgrad(self.ctx._h, D, H, W, _p(self.acts[l]), _p(g),
                                                     _p(self.gw[l]), _p(self.gb[l])))
            if l > 0:
                gn = self.g16[(LAYERS - l) % 2]
                # input gradient, masked by the ReLU of the layer input
                self._check(self.lib.mamute_conv3d(self.ctx._h, D, H, W, _p(g), _p(self.wb[l]),
                                                   None, 0, _p(self.acts[l]), None, _p(gn)))
                g = gn
        return loss.value

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        for l in range(LAYERS):
            self._check(self.lib.mamute_adam(self.ctx._h, self.w[l].numel(), _p(self.w[l]),
                                             _p(self.mw[l]), _p(self.vw[l]), _p(self.gw[l]), lr, b1,
                                             b2, eps, self.step))
            self._check(self.lib.mamute_adam(self.ctx._h, self.b[l].numel(), _p(self.b[l]),
                                             _p(self.mb[l]), _p(self.vb[l]), _p(self.gb[l]), lr, b1,
                                             b2, eps, self.step))
        self.pack()

    def train_step(self, x16, target, mask=None, lr=1e-3):
        loss = self.loss_and_grads(x16, target, mask)
        self.adam(lr)
        return loss

    def weights(self):
        return ([w.cpu().numpy() for w in self.w], [b.cpu().numpy() for b in self.b])

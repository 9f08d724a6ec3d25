"""Training data, training and evaluation of the learned GN-diagonal network.

Labels are the exact Gauss-Newton diagonal H (mamute_gn_diagonal) of
seeded models of the layered family, each smoothed by a random Gaussian
blur so that the inputs look like FWI iterates; the network input is the
velocity and the source-side pseudo-Hessian P (mamute_model with the
pseudo-Hessian output).  The network predicts the log-ratio log(H / P)
minus its training-set mean (net.offset), i.e. the receiver-side factor the
pseudo-Hessian lacks; the prediction is H^ = P exp(out + offset).  All
propagation, label and network arithmetic runs in libmamute.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import cnn, mamute, synth


@dataclasses.dataclass
class Sample:
    x16: torch.Tensor      # network input [D][H][W][16] BF16 bits
    target: torch.Tensor   # log(H / P) - offset [D][H][W]
    mask: torch.Tensor     # voxels used by the loss [D][H][W]
    n_mask: float
    pmax: float
    vel: torch.Tensor
    phess: torch.Tensor
    hdiag: torch.Tensor


def shallow_mask(shape, skip_planes: int, device) -> torch.Tensor:
    """Voxels below the acquisition layer (the source and receiver nodes
    make H and P singular there)."""
    m = torch.ones(shape, dtype=torch.float32, device=device)
    m[:skip_planes] = 0.0
    return m


def make_sample(ctx: mamute.Context, net: cnn.Net, w, vel: np.ndarray, band_rel: float = 1e-4,
                skip_planes: int = 8) -> Sample:
    dev = torch.device("cuda", ctx.device)
    g = mamute.grid_of(w)
    v = torch.from_numpy(np.ascontiguousarray(vel, np.float32)).to(dev)
    seis = torch.empty((int(w.rec_offset[-1]), w.nt), device=dev)
    ph = torch.empty_like(v)
    ctx.model(g, v, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis, phess=ph)
    hd = torch.empty_like(v)
    ctx.gn_diagonal(g, v, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, hd, band_rel=band_rel)
    x16, tgt, pmax = net.features(v, ph, hd)
    mask = shallow_mask(v.shape, skip_planes, dev)
    return Sample(x16, tgt, mask, float(mask.sum().item()), pmax, v, ph, hd)


def dataset(ctx, net, workload_fn, model_ids, blur_max: float = 8.0, seed: int = 0,
            set_offset: bool = True):
    """Samples for the given model ids; workload_fn(model_id) -> Workload.
    With set_offset the network's offset becomes the mean masked log(H / P)
    of these samples; the targets are centred by the network's offset."""
    rng = np.random.default_rng(seed)
    out = []
    for mid in model_ids:
        w = workload_fn(mid)
        vel = synth.gaussian_blur(w.vel, float(rng.uniform(0.0, blur_max)))
        out.append(make_sample(ctx, net, w, vel))
    if set_offset:
        tot, cnt = 0.0, 0.0
        for s in out:  # host-side statistic of the label set
            t = s.target.cpu().numpy().astype(np.float64)
            m = s.mask.cpu().numpy() > 0
            tot += t[m].sum()
            cnt += m.sum()
        net.offset = tot / max(cnt, 1.0)
    for s in out:
        s.target.sub_(net.offset)
    return out


def train(net: cnn.Net, data, epochs: int, lr: float = 2e-3, seed: int = 0, log=None):
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(data))
        tot = 0.0
        for i in order:
            s = data[i]
            tot += net.train_step(s.x16, s.target, s.mask, lr=lr)
        hist.append(tot / len(data))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def predict(net: cnn.Net, x16: torch.Tensor, phess: torch.Tensor) -> torch.Tensor:
    """H^ = P exp(out + offset)."""
    out = net.forward(x16).detach()
    return phess * torch.exp(out + float(net.offset))


def log_errors(net: cnn.Net, data):
    """Masked RMS of log(H^ / H) for the network and for the pseudo-Hessian,
    each after removing its own mean over the model (the preconditioner is
    insensitive to a global scale, which the L-BFGS scaling absorbs)."""
    res = []
    for s in data:
        m = s.mask > 0
        lh = torch.log(s.hdiag.clamp_min(1e-30))
        ln = torch.log(predict(net, s.x16, s.phess).clamp_min(1e-30))
        lp = torch.log(s.phess.clamp_min(1e-30))
        e_net = (ln - lh)[m]
        e_p = (lp - lh)[m]
        e_net = e_net - e_net.mean()
        e_p = e_p - e_p.mean()
        res.append((float(torch.sqrt((e_net ** 2).mean())), float(torch.sqrt((e_p ** 2).mean()))))
    return res

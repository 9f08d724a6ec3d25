"""Full-waveform inversion driver (Algorithm 2) with diagonal preconditioning.

The optimizer is a bound-projected L-BFGS (the paper's L-BFGS-b with lower
and upper velocity bounds, Sec. 2.1 and Table 3): two-loop recursion with
the initial inverse Hessian H0 = gamma * diag(1 / (h + eps max h)), where h
is the preconditioning diagonal, projection onto [vmin, vmax] and Armijo
backtracking on the projected step.  Every misfit, gradient and
pseudo-Hessian comes from libmamute (mamute_gradient with the pseudo-Hessian
output, mamute_model with mamute_misfit_noalloc for line-search trials); the
host keeps the FP64 model vectors and the L-BFGS pairs.

Preconditioners:
  'none'     h = 1
  'pseudo'   h = P, the source-side pseudo-Hessian of the current model
  'learned'  h = H^, the network's Gauss-Newton diagonal predicted from
             (velocity, P); a learned step is accepted only if Armijo holds
             within `learned_backtracks` backtracks, otherwise the iteration
             falls back to the 'pseudo' step.
  'exact'    h = H, the exact Gauss-Newton diagonal of the current model
             (mamute_gn_diagonal; what the network approximates, at the cost
             of 2 + n_rec / n_src propagations per shot).
"""
from __future__ import annotations

import ctypes
import dataclasses
import time

import numpy as np
import torch

from . import mamute


@dataclasses.dataclass
class Result:
    vel: np.ndarray
    history: list  # (wall seconds, misfit, kind of step)
    n_gradients: int
    n_forward: int


class Problem:
    """A workload's observed data and acquisition bound to a context."""

    def __init__(self, ctx: mamute.Context, w, d_obs: torch.Tensor, vmin: float, vmax: float):
        self.ctx, self.w, self.d_obs = ctx, w, d_obs
        self.grid = mamute.grid_of(w)
        self.vmin, self.vmax = vmin, vmax
        self.dev = d_obs.device
        self.lib = ctx.lib
        self.lib.mamute_misfit_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_longlong, ctypes.c_void_p,
                                                   ctypes.POINTER(ctypes.c_double)]
        self.seis = torch.empty_like(d_obs)
        self.n_grad = 0
        self.n_fwd = 0

    def gradient(self, v: np.ndarray):
        vt = torch.from_numpy(v.astype(np.float32)).to(self.dev)
        g = torch.empty_like(vt)
        ph = torch.empty_like(vt)
        w = self.w
        J = self.ctx.gradient(self.grid, vt, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                              self.d_obs, g, phess=ph)
        self.n_grad += 1
        return J, g.cpu().numpy().astype(np.float64).ravel(), ph

    def misfit(self, v: np.ndarray) -> float:
        vt = torch.from_numpy(v.astype(np.float32)).to(self.dev)
        w = self.w
        self.ctx.model(self.grid, vt, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                       self.seis)
        J = ctypes.c_double(0.0)
        stream = torch.cuda.current_stream(self.dev).cuda_stream
        rc = self.lib.mamute_misfit_noalloc(ctypes.c_void_p(self.seis.data_ptr()),
                                            ctypes.c_void_p(self.d_obs.data_ptr()),
                                            self.seis.numel(), ctypes.c_void_p(stream),
                                            ctypes.byref(J))
        if rc != mamute.OK:
            raise mamute.MamuteError(rc, "misfit")
        self.n_fwd += 1
        return J.value

    def project(self, v):
        return np.clip(v, self.vmin, self.vmax)


def two_loop(g, pairs, diag):
    """L-BFGS two-loop recursion with H0 = gamma * diag (Nocedal and Wright,
    Algorithm 7.4), gamma from the latest pair."""
    q = g.copy()
    alphas = []
    for s, y, rho in reversed(pairs):
        a = rho * np.dot(s, q)
        alphas.append(a)
        q -= a * y
    if pairs:
        s, y, _ = pairs[-1]
        gamma = np.dot(s, y) / max(np.dot(y, diag * y), 1e-300)
    else:
        gamma = 1.0
    r = gamma * diag * q
    for (s, y, rho), a in zip(pairs, reversed(alphas)):
        b = rho * np.dot(y, r)
        r += s * (a - b)
    return -r


def _diag(h, water=0.05):
    h = np.asarray(h, np.float64).ravel()
    return 1.0 / (h + water * h.max())


def _save_state(ckpt, it, x, J, g, ph, pairs, hist):
    arrays = {"x": x, "g": g, "ph": ph.detach().cpu().numpy()}
    for k, (s, y, _) in enumerate(pairs):
        arrays[f"s{k}"], arrays[f"y{k}"] = s, y
    ckpt.save(arrays, {"iteration": it, "J": J, "n_pairs": len(pairs),
                       "rho": [r for _, _, r in pairs], "history": hist})


def _load_state(ckpt, dev):
    got = ckpt.load()
    if got is None:
        return None
    a, m = got
    pairs = [(a[f"s{k}"], a[f"y{k}"], m["rho"][k]) for k in range(m["n_pairs"])]
    ph = torch.from_numpy(a["ph"]).to(dev)
    hist = [tuple(h) for h in m["history"]]
    return m["iteration"], a["x"], m["J"], a["g"], ph, pairs, hist


def run(prob: Problem, v0: np.ndarray, n_iter: int, precond: str = "pseudo", net=None,
        memory: int = 5, first_step: float = 40.0, learned_backtracks: int = 4,
        max_backtracks: int = 8, c1: float = 1e-4, water: float = 0.05,
        checkpoint: str | None = None, on_iteration=None) -> Result:
    """Projected L-BFGS on the misfit.  first_step (m/s) scales the first
    direction; later iterations try the unit L-BFGS step first.

    checkpoint: path of an optimizer-state file (resilience.Checkpoint).  The
    state (model, misfit, gradient, pseudo-Hessian, L-BFGS pairs, iteration,
    history) is written after every iteration; if the file exists when the
    run starts, the run resumes from it instead of starting from v0, and a
    resumed run ends with the same model as an uninterrupted one.
    on_iteration(it, x, J): called after iteration `it` has been saved."""
    shape = v0.shape
    ckpt = None
    state = None
    if checkpoint is not None:
        from .resilience import Checkpoint
        ckpt = Checkpoint(checkpoint)
        state = _load_state(ckpt, prob.dev)
    t0 = time.perf_counter()
    if state is not None:
        it0, x, J, g, ph, pairs, hist = state
        x = np.asarray(x, np.float64)
    else:
        it0 = 0
        x = prob.project(np.asarray(v0, np.float64).ravel())
        J, g, ph = prob.gradient(x.reshape(shape))
        hist = [(time.perf_counter() - t0, J, "start")]
        pairs = []
        if ckpt is not None:
            _save_state(ckpt, 0, x, J, g, ph, pairs, hist)

    def diag_for(kind, x, ph):
        if kind == "none":
            return np.ones_like(x)
        if kind == "pseudo":
            return _diag(ph.cpu().numpy(), water)
        if kind == "exact":
            vt = torch.from_numpy(x.reshape(shape).astype(np.float32)).to(prob.dev)
            hd = torch.empty_like(vt)
            w = prob.w
            prob.ctx.gn_diagonal(prob.grid, vt, None, w.src_xyz, w.wavelet, w.rec_offset,
                                 w.rec_xyz, hd)
            return _diag(hd.cpu().numpy(), water)
        vt = torch.from_numpy(x.reshape(shape).astype(np.float32)).to(prob.dev)
        x16, _, _ = net.features(vt, ph)
        out = net.forward(x16).cpu().numpy().astype(np.float64)
        return _diag(ph.cpu().numpy().astype(np.float64) * np.exp(out + net.offset), water)

    def line_search(d, J, g, x, max_bt, alpha, expand):
        for _ in range(max_bt + 1):
            xn = prob.project(x + alpha * d)
            Jn = prob.misfit(xn.reshape(shape))
            if Jn <= J + c1 * np.dot(g, xn - x):
                # without curvature information, grow the step while it pays
                for _ in range(4 if expand else 0):
                    xe = prob.project(x + 2.0 * alpha * d)
                    Je = prob.misfit(xe.reshape(shape))
                    if Je >= Jn:
                        break
                    xn, Jn, alpha = xe, Je, 2.0 * alpha
                return xn, Jn
            alpha *= 0.5
        return None, None

    for it in range(it0, n_iter):
        kinds = ["learned", "pseudo"] if precond == "learned" else [precond]
        accepted = None
        for kind in kinds:
            dg = diag_for(kind, x, ph)
            # Each kind restarts its own view of the memory when its direction
            # is not a descent direction, so a rejected learned attempt does
            # not change the fallback step; the shared memory is cleared only
            # if the accepted kind restarted it.
            mem = pairs
            d = two_loop(g, mem, dg)
            if np.dot(d, g) >= 0:  # not a descent direction: restart the memory
                mem = []
                d = two_loop(g, mem, dg)
            alpha = first_step / max(np.abs(d).max(), 1e-30) if not mem else 1.0
            nb = learned_backtracks if (kind == "learned") else max_backtracks
            xn, Jn = line_search(d, J, g, x, nb, alpha, expand=not mem)
            if xn is not None:
                accepted = (kind, xn, Jn)
                pairs = mem
                break
        if accepted is None:
            hist.append((time.perf_counter() - t0, J, "stalled"))
            break
        kind, xn, _ = accepted
        # The line search's misfits come from the allocation-free reduction,
        # which sums the residuals in the same order as the gradient call.
        Jn, gn, ph = prob.gradient(xn.reshape(shape))
        s, y = xn - x, gn - g
        sy = np.dot(s, y)
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            pairs.append((s, y, 1.0 / sy))
            pairs = pairs[-memory:]
        x, J, g = xn, Jn, gn
        hist.append((time.perf_counter() - t0, J, kind))
        if ckpt is not None:
            _save_state(ckpt, it + 1, x, J, g, ph, pairs, hist)
        if on_iteration is not None:
            on_iteration(it + 1, x, J)
    return Result(x.reshape(shape), hist, prob.n_grad, prob.n_fwd)

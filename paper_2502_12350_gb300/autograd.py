"""torch.autograd binding of the propagator.

forward(vel)  -> seismograms [n_rec][nt]         (mamute_model)
backward(g)   -> d<seis(vel), g>/d vel           (mamute_adjoint: adjoint
                 wavefield driven by g, cross-correlation imaging, with the
                 forward wavefield recomputed from revolve checkpoints held in
                 HBM; the adjoint-state method of Sec. 2.1 / Algorithm 3)

Density (if given) is a fixed parameter: no gradient flows to it.
"""
from __future__ import annotations

import torch

from . import mamute


class Acquisition:
    """Grid and acquisition of a modelling problem (host-side geometry)."""

    def __init__(self, grid: mamute.Grid, src_xyz, wavelet, rec_offset, rec_xyz, aperture=None,
                 n_snapshots: int = 0, check_mem: float = 0.8):
        self.grid = grid
        self.src_xyz = src_xyz
        self.wavelet = wavelet
        self.rec_offset = rec_offset
        self.rec_xyz = rec_xyz
        self.aperture = aperture
        self.n_snapshots = n_snapshots
        self.check_mem = check_mem

    @property
    def n_rec(self) -> int:
        return int(self.rec_offset[-1])


class _Propagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel, rho, acq: Acquisition, lib_ctx: mamute.Context):
        vel = vel.contiguous()
        seis = torch.empty((acq.n_rec, acq.grid.nt), device=vel.device, dtype=torch.float32)
        lib_ctx.model(acq.grid, vel, rho, acq.src_xyz, acq.wavelet, acq.rec_offset, acq.rec_xyz,
                      seis, aperture=acq.aperture)
        ctx.save_for_backward(vel, rho)
        ctx.acq = acq
        ctx.lib_ctx = lib_ctx
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        vel, rho = ctx.saved_tensors
        acq = ctx.acq
        grad = torch.empty_like(vel)
        ctx.lib_ctx.adjoint(acq.grid, vel, rho, acq.src_xyz, acq.wavelet, acq.rec_offset,
                            acq.rec_xyz, grad_seis.contiguous().float(), grad,
                            aperture=acq.aperture, n_snapshots=acq.n_snapshots,
                            check_mem=acq.check_mem)
        return grad, None, None, None


def propagate(vel: torch.Tensor, acq: Acquisition, lib_ctx: mamute.Context,
              rho: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable seismic modelling: seismograms as a function of vel."""
    return _Propagate.apply(vel, rho, acq, lib_ctx)

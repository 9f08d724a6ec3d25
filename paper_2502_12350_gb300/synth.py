"""Seeded synthetic inputs: velocity and density models, wavelets, acquisition.

This module holds input generation only (none of the propagator, adjoint or
imaging arithmetic), so both the CUDA path and the oracle may draw from it.
The model family follows the paper's synthetic-model scripts (Sec. 2.2.2:
constant, centred sphere and Gaussian models, Gardner density) and the
illustrative example (Sec. 3, Eq. 2); the seeded layered family with
Gaussian anomalies stands in for field models, since the paper uses no
public dataset.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea and Flood 2014), used to derive seeds."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def rng_for(config: int, model_id: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(splitmix64(1000 * config + model_id)))


def ricker(nt: int, dt: float, fpeak: float, amplitude: float = 1.0) -> np.ndarray:
    """Ricker wavelet w(t) = a (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
    tau = n dt - 1/f (the source signature of Sec. 3)."""
    tau = np.arange(nt, dtype=np.float64) * dt - 1.0 / fpeak
    arg = (math.pi * fpeak * tau) ** 2
    return (amplitude * (1.0 - 2.0 * arg) * np.exp(-arg)).astype(np.float32)


def gardner_density(vel: np.ndarray) -> np.ndarray:
    """Gardner's relation rho = 310 c^0.25 (kg/m^3, c in m/s), the density
    script of Sec. 2.2.2."""
    return (310.0 * np.power(vel.astype(np.float64), 0.25)).astype(np.float32)


def two_layer(nx, ny, nz, v_top=2000.0, v_bottom=3000.0, z_interface=32) -> np.ndarray:
    vel = np.full((nz, ny, nx), v_top, dtype=np.float32)
    vel[z_interface:] = v_bottom
    return vel


def gaussian_sphere(n=25, v_background=2500.0, v_peak=3500.0, sigma=3.0) -> np.ndarray:
    """Eq. 2 (Sec. 3): background plus a centred Gaussian of peak v_peak."""
    i = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    r2 = (x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2
    return (v_background + (v_peak - v_background) * np.exp(-0.5 * r2 / sigma**2)).astype(np.float32)


def layered_model(nx, ny, nz, rng: np.random.Generator, vmin=1500.0, vmax=4500.0) -> np.ndarray:
    """Seeded layered model: 4-8 layers with dipping (<= 3 deg) interfaces,
    velocities increasing with depth in [vmin, vmax], times 1-3 Gaussian
    anomalies of +/-10 %."""
    n_layers = int(rng.integers(4, 9))
    depths = np.sort(rng.uniform(0.05, 0.95, n_layers - 1)) * nz
    dips = np.radians(rng.uniform(0.0, 3.0, n_layers - 1))
    azim = rng.uniform(0.0, 2 * math.pi, n_layers - 1)
    vels = np.sort(rng.uniform(vmin, vmax, n_layers))
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    vel = np.full((nz, ny, nx), vels[0])
    for l in range(n_layers - 1):
        iface = depths[l] + math.tan(dips[l]) * (math.cos(azim[l]) * (x - nx / 2) +
                                                 math.sin(azim[l]) * (y - ny / 2))
        vel = np.where(z >= iface, vels[l + 1], vel)
    n_anom = int(rng.integers(1, 4))
    for _ in range(n_anom):
        amp = rng.uniform(-0.1, 0.1)
        sig = rng.uniform(0.05, 0.15, 3) * np.array([nx, ny, nz])
        cen = rng.uniform(0.2, 0.8, 3) * np.array([nx, ny, nz])
        r2 = ((x - cen[0]) / sig[0]) ** 2 + ((y - cen[1]) / sig[1]) ** 2 + ((z - cen[2]) / sig[2]) ** 2
        vel = vel * (1.0 + amp * np.exp(-0.5 * r2))
    return vel.astype(np.float32)


def gaussian_blur(vel: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Separable Gaussian smoothing with edge replication (initial models)."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(vel.astype(np.float64), sigma_cells, mode="nearest").astype(np.float32)


@dataclasses.dataclass
class Workload:
    """One synthetic problem: model, grid and acquisition in the API's units."""
    name: str
    nx: int
    ny: int
    nz: int
    border: int
    h: float
    dt: float
    nt: int
    fpeak: float
    vel: np.ndarray
    rho: np.ndarray | None
    src_xyz: np.ndarray        # [n_src][3] metres
    rec_offset: np.ndarray     # [n_src+1] int32
    rec_xyz: np.ndarray        # [total_rec][3] metres
    wavelet: np.ndarray        # [nt]
    aperture: np.ndarray | None = None   # [n_src][4] model cells (x0, x1, y0, y1)
    vel_init: np.ndarray | None = None

    @property
    def n_src(self):
        return len(self.src_xyz)

    @property
    def padded(self):
        b = 2 * self.border
        return (self.nz + b, self.ny + b, self.nx + b)

    @property
    def n_padded(self):
        z, y, x = self.padded
        return z * y * x


def _nodes_to_xyz(ix, iy, iz, h):
    return np.stack([np.asarray(ix, np.float64) * h, np.asarray(iy, np.float64) * h,
                     np.asarray(iz, np.float64) * h], axis=-1).reshape(-1, 3).astype(np.float32)


def forward_small(nt: int = 500, n: int = 64) -> Workload:
    """Forward modelling, constant density: 64^3, h = 10 m, dt = 1 ms, 500
    steps, 2000 m/s over 3000 m/s at z = 32, 16-cell sponge, Ricker 15 Hz at
    (32, 32, 8), 64 receivers on a line at z = 4."""
    h, dt = 10.0, 1e-3
    vel = two_layer(n, n, n, z_interface=n // 2)
    src = _nodes_to_xyz([n // 2], [n // 2], [8], h)
    rec = _nodes_to_xyz(np.arange(n), np.full(n, n // 2), np.full(n, 4), h)
    return Workload("forward_64cube_const_density", n, n, n, 16, h, dt, nt, 15.0, vel, None,
                    src, np.array([0, len(rec)], np.int32), rec, ricker(nt, dt, 15.0))


def forward_density(nt: int = 4000, nx=512, ny=512, nz=256, rec_step=2) -> Workload:
    """Forward modelling with density: 512x512x256, h = 12.5 m, dt = 1 ms,
    4000 steps, seeded layered model with anomalies and Gardner density,
    32-cell sponge, Ricker 10 Hz at (256, 256, 8), 256x256 receivers
    every 2 cells at z = 4."""
    h, dt = 12.5, 1e-3
    vel = layered_model(nx, ny, nz, rng_for(2, 0))
    rho = gardner_density(vel)
    src = _nodes_to_xyz([nx // 2], [ny // 2], [8], h)
    gx, gy = np.meshgrid(np.arange(0, nx, rec_step), np.arange(0, ny, rec_step), indexing="xy")
    rec = _nodes_to_xyz(gx.ravel(), gy.ravel(), np.full(gx.size, 4), h)
    return Workload(f"forward_{nx}x{ny}x{nz}_density", nx, ny, nz, 32, h, dt, nt, 10.0, vel, rho,
                    src, np.array([0, len(rec)], np.int32), rec, ricker(nt, dt, 10.0))


def gradient_single(nt: int = 2000, n: int = 256, rec_step: int = 2, border: int = 32) -> Workload:
    """Single-shot gradient: 256^3, h = 15 m, dt = 1.2 ms, 2000 steps, seeded
    layered model (true) and its Gaussian-smoothed version (initial,
    sigma = 1 % of the extent), Ricker 10 Hz at (128, 128, 8), 128x128
    receivers every 2 cells at z = 4, constant density."""
    h, dt = 15.0, 1.2e-3
    vel = layered_model(n, n, n, rng_for(3, 0))
    init = gaussian_blur(vel, 0.01 * n)
    src = _nodes_to_xyz([n // 2], [n // 2], [8], h)
    g = np.arange(0, n, rec_step)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    rec = _nodes_to_xyz(gx.ravel(), gy.ravel(), np.full(gx.size, 4), h)
    return Workload(f"gradient_{n}cube", n, n, n, border, h, dt, nt, 10.0, vel, None, src,
                    np.array([0, len(rec)], np.int32), rec, ricker(nt, dt, 10.0), vel_init=init)


def batched_shots(nt: int = 2500, nx=600, ny=600, nz=200, n_side=8, rec_side=96,
                  ap_min=128, ap_max=320, border=20, seed_cfg=4) -> Workload:
    """Batched gradient: 64 shots on an 8x8 grid at z = 4 over a 600x600x200
    model (h = 15 m, dt = 1.2 ms, Ricker 8 Hz); each shot owns an aperture
    of U{128..320} cells per lateral axis centred on the source and clipped
    to the model, with 96x96 receivers spread across it at z = 4."""
    h, dt = 15.0, 1.2e-3
    rng = rng_for(seed_cfg, 1)
    vel = layered_model(nx, ny, nz, rng_for(seed_cfg, 0))
    init = gaussian_blur(vel, 8.0)
    srcs, recs, offs, aps = [], [], [0], []
    for j in range(n_side):
        for i in range(n_side):
            sx = int(round((i + 0.5) * nx / n_side))
            sy = int(round((j + 0.5) * ny / n_side))
            lx, ly = (int(v) for v in rng.integers(ap_min, ap_max + 1, 2))
            x0 = max(0, min(nx - lx, sx - lx // 2)) if lx < nx else 0
            x0 -= x0 % 4  # window x origin on a 16-byte boundary
            y0 = max(0, min(ny - ly, sy - ly // 2)) if ly < ny else 0
            x1, y1 = min(nx, x0 + lx), min(ny, y0 + ly)
            aps.append((x0, x1, y0, y1))
            srcs.append((sx, sy, 4))
            rx = np.unique(np.linspace(x0, x1 - 1, rec_side).round().astype(int))
            ry = np.unique(np.linspace(y0, y1 - 1, rec_side).round().astype(int))
            gx, gy = np.meshgrid(rx, ry, indexing="xy")
            recs.append(_nodes_to_xyz(gx.ravel(), gy.ravel(), np.full(gx.size, 4), h))
            offs.append(offs[-1] + gx.size)
    src = _nodes_to_xyz([s[0] for s in srcs], [s[1] for s in srcs], [s[2] for s in srcs], h)
    return Workload(f"batched_{n_side * n_side}shots_{nx}x{ny}x{nz}", nx, ny, nz, border, h, dt,
                    nt, 8.0, vel, None, src, np.array(offs, np.int32), np.concatenate(recs),
                    ricker(nt, dt, 8.0), aperture=np.array(aps, np.int32), vel_init=init)


def fwi_small(model_id: int = 0, nt: int = 1500, nx=160, ny=160, nz=80, border=20) -> Workload:
    """Learned-preconditioner FWI workload: 160x160x80 (h = 15 m, dt =
    1.2 ms, 1500 steps), 12 shots on a 4x3 grid and 64 receivers (8x8) at
    z = 4, Ricker 8 Hz; the initial model is the true one blurred with
    sigma = 8 cells."""
    h, dt = 15.0, 1.2e-3
    vel = layered_model(nx, ny, nz, rng_for(5, model_id))
    init = gaussian_blur(vel, 8.0)
    sx = [int(round((i + 0.5) * nx / 4)) for j in range(3) for i in range(4)]
    sy = [int(round((j + 0.5) * ny / 3)) for j in range(3) for i in range(4)]
    src = _nodes_to_xyz(sx, sy, [4] * 12, h)
    r = np.linspace(4, nx - 5, 8).round().astype(int)
    gx, gy = np.meshgrid(r, np.linspace(4, ny - 5, 8).round().astype(int), indexing="xy")
    one = _nodes_to_xyz(gx.ravel(), gy.ravel(), np.full(gx.size, 4), h)
    rec = np.concatenate([one] * 12)
    offs = np.arange(13, dtype=np.int32) * len(one)
    return Workload(f"fwi_{nx}x{ny}x{nz}_m{model_id}", nx, ny, nz, border, h, dt, nt, 8.0, vel, None,
                    src, offs, rec, ricker(nt, dt, 8.0), vel_init=init)


def small_case(seed: int = 0, nx=24, ny=20, nz=18, border=8, nt=60, density=True, n_src=2,
               n_rec=7, h=10.0, dt=1e-3, fpeak=25.0) -> Workload:
    """Small ragged random case for parity tests: odd sizes, several shots,
    receivers scattered through the model (including duplicated nodes)."""
    rng = np.random.Generator(np.random.PCG64(splitmix64(7919 + seed)))
    vel = layered_model(nx, ny, nz, rng, vmin=1800.0, vmax=3200.0)
    rho = gardner_density(vel) if density else None
    src = np.stack([rng.integers(0, nx, n_src), rng.integers(0, ny, n_src),
                    rng.integers(0, nz, n_src)], axis=1)
    src_xyz = (src * h).astype(np.float32)
    recs, offs = [], [0]
    for s in range(n_src):
        r = np.stack([rng.integers(0, nx, n_rec), rng.integers(0, ny, n_rec),
                      rng.integers(0, nz, n_rec)], axis=1)
        r[-1] = r[0]  # a duplicated receiver node
        recs.append((r * h).astype(np.float32))
        offs.append(offs[-1] + n_rec)
    return Workload(f"small_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz, border, h, dt, nt, fpeak, vel, rho,
                    src_xyz, np.array(offs, np.int32), np.concatenate(recs),
                    ricker(nt, dt, fpeak))

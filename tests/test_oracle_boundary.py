"""Pins of the oracle's free surface (image method) and trilinear off-grid
sources and receivers (Sec. 2: modelling with a free surface; source and
receiver positions in metres).

* The free surface is pinned by the image-source identity: with no sponge,
  a run with the top model plane as a pressure-release surface equals a run
  on the model mirrored about that plane (no free surface) driven by the
  source and an opposite-sign image source, exactly.
* The trilinear points are pinned by linearity: data of an off-grid receiver
  (or source) is the weighted sum of the data of nearest-node runs at the 8
  surrounding nodes, with the weights written out here.
* Both keep the adjoint dot-product identity.
"""
import itertools

import numpy as np
import pytest

from paper_2502_12350_gb300 import synth


def _model(seed, nx, ny, nz):
    rng = np.random.default_rng(seed)
    return rng.uniform(1900.0, 2600.0, (nz, ny, nx))


@pytest.mark.parametrize("density", [False, True])
def test_free_surface_equals_odd_image_source(oracle, density):
    nx, ny, nz, b, h, dt, nt = 11, 10, 9, 4, 10.0, 1e-3, 60
    vel = _model(1, nx, ny, nz)
    rho = None
    if density:  # varies laterally only, so it is the same under the mirror
        rng = np.random.default_rng(2)
        rho = np.broadcast_to(rng.uniform(1800, 2600, (1, ny, nx)), (nz, ny, nx)).copy()
    w = synth.ricker(nt, dt, 35.0).astype(np.float64)
    src = np.array([[5 * h, 4 * h, 3 * h]])
    rec = np.array([[2 * h, 7 * h, 1 * h], [8 * h, 3 * h, 5 * h], [5 * h, 4 * h, 8 * h]])
    g_fs = oracle.make_grid(nx, ny, nz, b, h, dt, nt, cerjan=0.0, free_surface=1)
    d_fs = oracle.model(g_fs, vel, src, w, [0, 3], rec, rho=rho)
    # mirrored model: plane k of the free-surface run is plane k + nz - 1 here
    nzd = 2 * nz - 1
    mirror = np.concatenate([vel[:0:-1], vel], axis=0)
    rho_d = None if rho is None else np.concatenate([rho[:0:-1], rho], axis=0)
    assert mirror.shape[0] == nzd
    g_d = oracle.make_grid(nx, ny, nzd, b, h, dt, nt, cerjan=0.0)
    shift = np.array([0.0, 0.0, (nz - 1) * h])
    img = src.copy()
    img[0, 2] = (nz - 1) * h - src[0, 2]  # mirror image of the source depth
    d_src = oracle.model(g_d, mirror, src + shift, w, [0, 3], rec + shift, rho=rho_d)
    d_img = oracle.model(g_d, mirror, img, w, [0, 3], rec + shift, rho=rho_d)
    ref = d_src - d_img
    assert np.abs(d_fs).max() > 0
    np.testing.assert_allclose(d_fs, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # and it is not the run without the surface
    g_0 = oracle.make_grid(nx, ny, nz, b, h, dt, nt, cerjan=0.0)
    d_0 = oracle.model(g_0, vel, src, w, [0, 3], rec, rho=rho)
    assert np.abs(d_0 - d_fs).max() > 1e-3 * np.abs(d_fs).max()


def test_free_surface_rejects_points_on_the_surface(oracle):
    nx, ny, nz = 8, 8, 8
    g = oracle.make_grid(nx, ny, nz, 3, 10.0, 1e-3, 10, free_surface=1)
    vel = np.full((nz, ny, nx), 2000.0)
    w = np.ones(10)
    with pytest.raises(ValueError):
        oracle.model(g, vel, [[40.0, 40.0, 0.0]], w, [0, 1], [[40.0, 40.0, 30.0]])
    with pytest.raises(ValueError):
        oracle.model(g, vel, [[40.0, 40.0, 30.0]], w, [0, 1], [[40.0, 40.0, 0.0]])


def _weights(frac):
    """Trilinear weights of the 8 corners (dx, dy, dz in {0, 1}) of a cell."""
    tx, ty, tz = frac
    return {(i, j, k): (tx if i else 1 - tx) * (ty if j else 1 - ty) * (tz if k else 1 - tz)
            for i, j, k in itertools.product((0, 1), repeat=3)}


@pytest.mark.parametrize("density", [False, True])
def test_trilinear_receiver_and_source_are_weighted_node_sums(oracle, density):
    w8 = synth.small_case(seed=61, nx=12, ny=11, nz=10, border=4, nt=45, density=density,
                          n_src=1, n_rec=1, fpeak=35.0)
    h = w8.h
    vel = w8.vel.astype(np.float64)
    rho = None if w8.rho is None else w8.rho.astype(np.float64)
    base, frac = np.array([4, 5, 3]), np.array([0.3, 0.75, 0.55])
    x_off = (base + frac) * h
    node = lambda c: ((base + np.array(c)) * h)[None, :]
    src_on = np.array([[8 * h, 2 * h, 6 * h]])
    gt = oracle.make_grid(w8.nx, w8.ny, w8.nz, w8.border, h, w8.dt, w8.nt, xyz_interp=1)
    gn = oracle.make_grid(w8.nx, w8.ny, w8.nz, w8.border, h, w8.dt, w8.nt, xyz_interp=0)
    wts = _weights(frac)
    # receiver off the grid
    got = oracle.model(gt, vel, src_on, w8.wavelet, [0, 1], x_off[None, :], rho=rho)
    ref = sum(wt * oracle.model(gn, vel, src_on, w8.wavelet, [0, 1], node(c), rho=rho)
              for c, wt in wts.items())
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # source off the grid
    got = oracle.model(gt, vel, x_off[None, :], w8.wavelet, [0, 1], src_on, rho=rho)
    ref = sum(wt * oracle.model(gn, vel, node(c), w8.wavelet, [0, 1], src_on, rho=rho)
              for c, wt in wts.items())
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # on-grid coordinates give the nearest-node result bit for bit
    on = oracle.model(gt, vel, src_on, w8.wavelet, [0, 1], node((1, 0, 1)), rho=rho)
    np.testing.assert_array_equal(on, oracle.model(gn, vel, src_on, w8.wavelet, [0, 1],
                                                   node((1, 0, 1)), rho=rho))


@pytest.mark.parametrize("free_surface,xyz_interp", [(1, 0), (0, 1), (1, 1)])
def test_dot_product_with_surface_and_offgrid_points(oracle, free_surface, xyz_interp):
    w = synth.small_case(seed=62, nx=12, ny=11, nz=10, border=5, nt=40, density=True, n_src=2,
                         n_rec=5, fpeak=30.0)
    rng = np.random.default_rng(9)
    # off-grid positions at depth >= 1 cell (below a free surface)
    w.src_xyz = (w.src_xyz + rng.uniform(0.1, 0.9, w.src_xyz.shape) * w.h).astype(np.float64)
    w.rec_xyz = (w.rec_xyz + rng.uniform(0.1, 0.9, w.rec_xyz.shape) * w.h).astype(np.float64)
    lim = np.array([w.nx - 1, w.ny - 1, w.nz - 1]) * w.h - 1e-6
    w.src_xyz = np.clip(w.src_xyz, w.h, lim)
    w.rec_xyz = np.clip(w.rec_xyz, w.h, lim)
    if not xyz_interp:
        w.src_xyz = np.round(w.src_xyz / w.h) * w.h
        w.rec_xyz = np.round(w.rec_xyz / w.h) * w.h
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt,
                         free_surface=free_surface, xyz_interp=xyz_interp)
    wav = rng.standard_normal(w.nt)
    r = rng.standard_normal((int(w.rec_offset[-1]), w.nt))
    Fw = oracle.model(g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, rho=w.rho)
    _, _, FTr = oracle.gradient(g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, Fw - r,
                                rho=w.rho, return_dwav=True)
    w2 = rng.standard_normal(w.nt)
    Fw2 = oracle.model(g, w.vel, w.src_xyz, w2, w.rec_offset, w.rec_xyz, rho=w.rho)
    lhs, rhs = np.sum(Fw2 * r), np.sum(w2 * FTr)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_gradient_fd_with_free_surface_and_offgrid_points(oracle):
    w = synth.small_case(seed=63, nx=10, ny=9, nz=9, border=4, nt=40, density=True, n_src=1,
                         n_rec=4, fpeak=35.0)
    rng = np.random.default_rng(10)
    w.src_xyz = np.array([[4.4 * w.h, 3.7 * w.h, 2.5 * w.h]])
    w.rec_xyz = np.array([[1.2 * w.h, 2.6 * w.h, 1.5 * w.h], [7.3 * w.h, 5.1 * w.h, 1.1 * w.h],
                          [5.5 * w.h, 7.9 * w.h, 6.2 * w.h], [2.0 * w.h, 6.0 * w.h, 3.0 * w.h]])
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, free_surface=1,
                         xyz_interp=1)
    vel = w.vel.astype(np.float64)
    dobs = oracle.model(g, vel * (1 + 0.03 * rng.standard_normal(vel.shape)), w.src_xyz,
                        w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    _, grad = oracle.gradient(g, vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                              rho=w.rho)
    dc = np.zeros_like(vel)
    dc[1:-1, 1:-1, 1:-1] = rng.standard_normal(tuple(s - 2 for s in vel.shape)) * 50.0

    def J(v):
        d = oracle.model(g, v, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
        return 0.5 * np.sum((d - dobs) ** 2)

    pred = np.sum(grad * dc)
    eps = 1e-3
    fd = (J(vel + eps * dc) - J(vel - eps * dc)) / (2 * eps)
    assert abs(fd - pred) <= 1e-6 * abs(pred)

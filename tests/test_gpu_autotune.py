"""The measured autotuner: it caches a valid decomposition for the problem
shape, a second call reuses the cache, and the seismograms do not depend on
the decomposition."""
import json

import numpy as np
import pytest

from paper_2502_12350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_caches_and_preserves_results(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import autotune, build, mamute
    build.build()
    monkeypatch.setenv("MAMUTE_AUTOTUNE_CACHE", str(tmp_path / "tiles.json"))
    ctx = mamute.Context(0)
    w = synth.small_case(seed=81, nx=60, ny=52, nz=40, border=8, nt=48, n_src=2, n_rec=10)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    rho = torch.from_numpy(w.rho).to(dev)
    g = mamute.grid_of(w)
    seis = torch.empty((int(w.rec_offset[-1]), w.nt), device=dev)
    ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis)
    ref = seis.cpu().numpy()
    tiles = autotune.tune_model(ctx, g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                                seis, steps=8, candidates=[(64, 16), (32, 8), (72, 16)])
    cache = json.load(open(tmp_path / "tiles.json"))
    assert len(cache) == 1 and list(cache.values())[0]["tiles"] == tiles
    assert tuple(tiles[:2]) in [(64, 16), (32, 8), (72, 16)] and tiles[2] >= 1
    again = autotune.tune_model(ctx, g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                                seis, steps=8, candidates=[(128, 8)])
    assert again == tiles  # served from the cache
    ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis, tiles=tiles)
    np.testing.assert_array_equal(seis.cpu().numpy(), ref)
    with pytest.raises(mamute.MamuteError):
        ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis,
                  tiles=[40, 40, 1, 0, 0, 0])
    ctx.close()


def test_gradient_autotune_preserves_gradient(tmp_path, monkeypatch):
    """Tuning the adjoint decomposition caches a choice and the gradient
    computed with it equals the default one bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import autotune, build, mamute
    build.build()
    monkeypatch.setenv("MAMUTE_AUTOTUNE_CACHE", str(tmp_path / "tiles.json"))
    ctx = mamute.Context(0)
    w = synth.small_case(seed=82, nx=60, ny=52, nz=40, border=8, nt=40, n_src=2, n_rec=10)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    rho = torch.from_numpy(w.rho).to(dev)
    g = mamute.grid_of(w)
    dobs = torch.zeros((int(w.rec_offset[-1]), w.nt), device=dev)
    ref = torch.empty_like(vel)
    J0 = ctx.gradient(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs, ref)
    tiles = autotune.tune_gradient(ctx, g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset,
                                   w.rec_xyz, dobs, n_snapshots=0, steps=8,
                                   candidates=[(64, 8), (32, 16), (72, 16)])
    assert tiles[:3] == [0, 0, 0] and tuple(tiles[3:5]) in [(64, 8), (32, 16), (72, 16)]
    assert len(json.load(open(tmp_path / "tiles.json"))) == 1
    grad = torch.empty_like(vel)
    J = ctx.gradient(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs, grad,
                     tiles=tiles)
    assert J == J0
    assert bool(torch.equal(grad, ref))
    ctx.close()

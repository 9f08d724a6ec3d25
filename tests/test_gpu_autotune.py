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

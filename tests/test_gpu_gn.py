"""GN-diagonal labels on the GPU against the oracle's separable form (same
band limit); the oracle's separable form is pinned to its brute-force
definition in test_oracle_gn.py."""
import numpy as np
import pytest

from oracle import gn
from paper_2502_12350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, mamute
    build.build()
    c = mamute.Context(0)
    yield c
    c.close()


def _common_receivers(density, seed, nt=120, nx=14, ny=12):
    w = synth.small_case(seed=seed, nx=nx, ny=ny, nz=10, border=6, nt=nt, density=density,
                         n_src=3, n_rec=5, fpeak=35.0)
    one = w.rec_xyz[:5]
    w.rec_xyz = np.concatenate([one] * w.n_src)
    w.rec_offset = np.arange(w.n_src + 1, dtype=np.int32) * 5
    return w


@pytest.mark.parametrize("density", [False, True])
def test_gn_diagonal_matches_oracle(ctx, oracle, density):
    from paper_2502_12350_gb300 import mamute
    w = _common_receivers(density, 61 + int(density))
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    ref = gn.separable(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       band_rel=1e-4)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    rho = None if w.rho is None else torch.from_numpy(w.rho).to(dev)
    H = torch.full_like(vel, float("nan"))
    ctx.gn_diagonal(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                    H, band_rel=1e-4)
    got = H.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all() and got.min() > 0
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3


def test_gn_rejects_differing_receivers(ctx):
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=63, nx=14, ny=12, nz=10, border=6, nt=40, n_src=2, n_rec=4)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    H = torch.empty_like(vel)
    with pytest.raises(mamute.MamuteError) as e:
        ctx.gn_diagonal(mamute.grid_of(w), vel, None, w.src_xyz, w.wavelet, w.rec_offset,
                        w.rec_xyz, H)
    assert e.value.code == mamute.EINVAL


def test_gn_diagonal_full_band(ctx, oracle):
    """All nt + 1 one-sided bins (the largest DFT configuration: 121 bins)."""
    from paper_2502_12350_gb300 import mamute
    w = _common_receivers(False, 64, nt=120)
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    ref = gn.separable(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    H = torch.full_like(vel, float("nan"))
    ctx.gn_diagonal(mamute.grid_of(w), vel, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                    H, band_rel=0.0)
    got = H.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3


@pytest.mark.parametrize("nt,nx,ny", [(300, 14, 12), (120, 13, 11)])
def test_gn_diagonal_blocks_and_fp32_path(ctx, oracle, nt, nx, ny):
    """nt = 300: two accumulation blocks on the tensor cores (256 samples and
    a ragged 44); 13 x 11 x 10 points (not a multiple of 4): the FP32 path."""
    from paper_2502_12350_gb300 import mamute
    w = _common_receivers(True, 65, nt=nt, nx=nx, ny=ny)
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    ref = gn.separable(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       band_rel=1e-4)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    rho = torch.from_numpy(w.rho).to(dev)
    H = torch.full_like(vel, float("nan"))
    ctx.gn_diagonal(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                    H, band_rel=1e-4)
    got = H.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all() and got.min() > 0
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3


@pytest.mark.parametrize("cap", [0, 4, 3])
def test_gn_receiver_batches_beyond_the_shots(ctx, oracle, monkeypatch, cap):
    """Receivers are batched independently of the shots: more receivers per
    launch than there are shot windows (a plan of their own), in one batch
    (no cap) or in several (batches of 4 and 3, and of 3, 3 and 1)."""
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=66, nx=14, ny=12, nz=10, border=6, nt=80, density=True, n_src=2,
                         n_rec=7, fpeak=35.0)
    w.rec_xyz = np.concatenate([w.rec_xyz[:7]] * 2)
    w.rec_offset = np.array([0, 7, 14], np.int32)
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    ref = gn.separable(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       band_rel=1e-4)
    monkeypatch.setenv("MAMUTE_GN_BATCH", str(cap))
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    H = torch.full_like(vel, float("nan"))
    ctx.gn_diagonal(mamute.grid_of(w), vel, torch.from_numpy(w.rho).to(dev), w.src_xyz,
                    w.wavelet, w.rec_offset, w.rec_xyz, H, band_rel=1e-4)
    got = H.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all() and got.min() > 0
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3

"""Parity of the free surface and of trilinear off-grid sources and receivers
(CUDA path through the C ABI) with the FP64 oracle, and their invariance
under the work decomposition."""
import numpy as np
import pytest

from paper_2502_12350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEIS_TOL_64 = 1e-4
SEIS_TOL_32 = 1e-5
GRAD_COS = 0.9999


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, mamute
    build.build()
    c = mamute.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def cosine(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return a @ b / (np.linalg.norm(a) * np.linalg.norm(b))


def _offgrid(w, seed, depth_min=1.0):
    """Moves sources and receivers off the grid (depth >= depth_min cells)."""
    rng = np.random.default_rng(seed)
    lim = np.array([w.nx - 1, w.ny - 1, w.nz - 1]) * w.h - 1e-3
    lo = np.array([0.0, 0.0, depth_min * w.h])
    w.src_xyz = np.clip(w.src_xyz + rng.uniform(0.05, 0.95, w.src_xyz.shape) * w.h, lo,
                        lim).astype(np.float32)
    w.rec_xyz = np.clip(w.rec_xyz + rng.uniform(0.05, 0.95, w.rec_xyz.shape) * w.h, lo,
                        lim).astype(np.float32)
    return w


def _below_surface(w):
    w.src_xyz = w.src_xyz.copy()
    w.rec_xyz = w.rec_xyz.copy()
    w.src_xyz[:, 2] = np.maximum(w.src_xyz[:, 2], w.h)
    w.rec_xyz[:, 2] = np.maximum(w.rec_xyz[:, 2], w.h)
    return w


def gpu_model(ctx, w, fs, xi, **opts):
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    seis = torch.full((int(w.rec_offset[-1]), w.nt), float("nan"), device=dev)
    ctx.model(mamute.grid_of(w, free_surface=fs, xyz_interp=xi), vel, rho, w.src_xyz, w.wavelet,
              w.rec_offset, w.rec_xyz, seis, aperture=w.aperture, **opts)
    return seis.cpu().numpy()


def gpu_gradient(ctx, w, dobs, fs, xi, **opts):
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(dobs, np.float32)).to(dev)
    grad = torch.full_like(vel, float("nan"))
    J = ctx.gradient(mamute.grid_of(w, free_surface=fs, xyz_interp=xi), vel, rho, w.src_xyz,
                     w.wavelet, w.rec_offset, w.rec_xyz, d, grad, aperture=w.aperture, **opts)
    return J, grad.cpu().numpy()


def ogrid(oracle, w, fs, xi):
    return oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, free_surface=fs,
                            xyz_interp=xi)


CASES = [
    (dict(seed=90, nx=30, ny=26, nz=22, border=6, nt=60, density=True, n_src=2, n_rec=9), 1, 0),
    (dict(seed=91, nx=37, ny=21, nz=19, border=5, nt=50, density=False, n_src=3, n_rec=7), 0, 1),
    (dict(seed=92, nx=29, ny=33, nz=17, border=7, nt=55, density=True, n_src=2, n_rec=8), 1, 1),
]


@pytest.mark.parametrize("case,fs,xi", CASES)
def test_model_matches_oracle(ctx, oracle, case, fs, xi):
    w = synth.small_case(**case)
    w = _offgrid(w, case["seed"]) if xi else _below_surface(w)
    got = gpu_model(ctx, w, fs, xi)
    og = ogrid(oracle, w, fs, xi)
    ref64 = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    ref32 = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                         precision=32)
    assert np.isfinite(got).all()
    assert rel(got, ref64) <= SEIS_TOL_64
    assert rel(got, ref32) <= SEIS_TOL_32


@pytest.mark.parametrize("case,fs,xi", CASES)
def test_gradient_matches_oracle(ctx, oracle, case, fs, xi):
    w = synth.small_case(**case)
    w = _offgrid(w, case["seed"]) if xi else _below_surface(w)
    og = ogrid(oracle, w, fs, xi)
    rng = np.random.default_rng(case["seed"])
    vtrue = (w.vel * (1 + 0.05 * rng.standard_normal(w.vel.shape))).astype(np.float32)
    dobs = oracle.model(og, vtrue, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                        rho=w.rho).astype(np.float32)
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                             rho=w.rho)
    for ns in (-1, 4):
        J, g = gpu_gradient(ctx, w, dobs, fs, xi, n_snapshots=ns)
        assert np.isfinite(g).all()
        assert cosine(g, gr) >= GRAD_COS
        assert abs(J - Jr) <= 1e-4 * Jr


def test_free_surface_bitwise_across_decompositions(ctx, monkeypatch):
    """The image planes come from the producer's plane map and the consumers'
    sign, so z blocks (primed from planes above the surface) and tile shapes
    change nothing."""
    w = _below_surface(synth.small_case(seed=93, nx=34, ny=30, nz=26, border=6, nt=40, n_src=2,
                                        n_rec=8))
    ref = gpu_model(ctx, w, 1, 0)
    dobs = np.zeros_like(ref)
    Jr, gr = gpu_gradient(ctx, w, dobs + 1e-3 * ref.max(), 1, 0, n_snapshots=3)
    for zs, tile in ((3, (64, 16)), (6, (32, 8)), (2, (128, 8))):
        monkeypatch.setenv("MAMUTE_ZSPLIT", str(zs))
        monkeypatch.setenv("MAMUTE_ADJ_ZSPLIT", str(zs))
        monkeypatch.setenv("MAMUTE_TX", str(tile[0]))
        monkeypatch.setenv("MAMUTE_TY", str(tile[1]))
        np.testing.assert_array_equal(gpu_model(ctx, w, 1, 0), ref)
        J, g = gpu_gradient(ctx, w, dobs + 1e-3 * ref.max(), 1, 0, n_snapshots=3)
        assert J == Jr
        np.testing.assert_array_equal(g, gr)


def test_offgrid_host_entry_point_and_apertures(ctx, oracle):
    """Trilinear receivers through the host entry point (segmented copies of
    the per-node sums) equal the device entry point; with apertures they
    match the oracle's windows."""
    from paper_2502_12350_gb300 import mamute
    w = _offgrid(synth.small_case(seed=94, nx=28, ny=24, nz=18, border=5, nt=64, n_src=2,
                                  n_rec=10), 94)
    dev_out = gpu_model(ctx, w, 0, 1)
    host_out = np.zeros_like(dev_out, dtype=np.float32)
    ctx.model_host(mamute.grid_of(w, xyz_interp=1), np.ascontiguousarray(w.vel),
                   np.ascontiguousarray(w.rho), w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                   host_out)
    np.testing.assert_array_equal(host_out, dev_out)
    # two shots, each in an aperture window holding all of its points
    w.aperture = np.array([[0, 20, 2, 22], [4, 28, 0, 24]], np.int32)
    for s in range(2):
        a = w.aperture[s]
        sl = slice(w.rec_offset[s], w.rec_offset[s + 1])
        w.rec_xyz[sl, 0] = np.clip(w.rec_xyz[sl, 0], a[0] * w.h, (a[1] - 1) * w.h - 1e-3)
        w.rec_xyz[sl, 1] = np.clip(w.rec_xyz[sl, 1], a[2] * w.h, (a[3] - 1) * w.h - 1e-3)
        w.src_xyz[s, 0] = np.clip(w.src_xyz[s, 0], a[0] * w.h, (a[1] - 1) * w.h - 1e-3)
        w.src_xyz[s, 1] = np.clip(w.src_xyz[s, 1], a[2] * w.h, (a[3] - 1) * w.h - 1e-3)
    got = gpu_model(ctx, w, 0, 1)
    ref = oracle.model(ogrid(oracle, w, 0, 1), w.vel, w.src_xyz, w.wavelet, w.rec_offset,
                       w.rec_xyz, rho=w.rho, aperture=w.aperture)
    assert rel(got, ref) <= SEIS_TOL_64


def test_points_on_the_free_surface_are_rejected(ctx):
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=95, nx=16, ny=16, nz=12, border=4, nt=10, n_src=1, n_rec=3)
    w.src_xyz = w.src_xyz.copy()
    w.src_xyz[0, 2] = 0.0
    with pytest.raises(mamute.MamuteError) as e:
        gpu_model(ctx, w, 1, 0)
    assert e.value.code == mamute.EINVAL

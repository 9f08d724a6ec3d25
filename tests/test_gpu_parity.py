"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: seismogram relative L2 <= 1e-4 against the FP64 oracle and
<= 1e-5 against the oracle's FP32 mode; gradient cosine >= 0.9999 and
misfit within 1e-4 relative.
"""
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


def gpu_model(ctx, w, **opts):
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    seis = torch.full((int(w.rec_offset[-1]), w.nt), float("nan"), device=dev)
    ctx.model(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis,
              aperture=w.aperture, **opts)
    return seis.cpu().numpy()


def gpu_gradient(ctx, w, dobs, **opts):
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(dobs, np.float32)).to(dev)
    grad = torch.full_like(vel, float("nan"))
    J = ctx.gradient(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                     d, grad, aperture=w.aperture, **opts)
    return J, grad.cpu().numpy()


def ogrid(oracle, w):
    return oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)


CASES = [
    dict(seed=0, nx=24, ny=20, nz=18, border=8, nt=60, density=True),
    dict(seed=1, nx=37, ny=29, nz=21, border=6, nt=70, density=False, n_src=3),
    dict(seed=2, nx=70, ny=19, nz=33, border=5, nt=50, density=True, n_src=1, n_rec=40),
    dict(seed=3, nx=9, ny=5, nz=6, border=3, nt=30, density=True),
]


@pytest.mark.parametrize("case", CASES)
def test_model_matches_oracle(ctx, oracle, case):
    w = synth.small_case(**case)
    got = gpu_model(ctx, w)
    og = ogrid(oracle, w)
    ref64 = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    ref32 = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                         precision=32)
    assert np.isfinite(got).all()
    assert rel(got, ref64) <= SEIS_TOL_64
    assert rel(got, ref32) <= SEIS_TOL_32


def test_model_forward_64cube_const_density(ctx, oracle):
    """The 64^3 two-layer workload (500 steps, 16-cell sponge, 64 receivers)."""
    w = synth.forward_small()
    got = gpu_model(ctx, w)
    ref = oracle.model(ogrid(oracle, w), w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz)
    assert rel(got, ref) <= SEIS_TOL_64


@pytest.mark.parametrize("tile", [(64, 16), (64, 8), (32, 16), (32, 8), (128, 8)])
def test_tiles_bitwise_identical(ctx, monkeypatch, tile):
    """The arithmetic per point does not depend on the tile shape."""
    w = synth.small_case(seed=4, nx=45, ny=33, nz=20, border=6, nt=40)
    ref = gpu_model(ctx, w)
    monkeypatch.setenv("MAMUTE_TX", str(tile[0]))
    monkeypatch.setenv("MAMUTE_TY", str(tile[1]))
    got = gpu_model(ctx, w)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("zsplit", [2, 3, 6])
def test_z_blocks_bitwise_identical(ctx, monkeypatch, zsplit):
    """Splitting the planes into z blocks (each primed from its neighbours'
    planes) changes nothing; the gradient too (adjoint z blocks)."""
    w = synth.small_case(seed=13, nx=30, ny=26, nz=28, border=6, nt=35, n_src=2, n_rec=8)
    ref = gpu_model(ctx, w)
    dobs = np.zeros_like(ref)
    Jr, gr = gpu_gradient(ctx, w, dobs, n_snapshots=3)
    monkeypatch.setenv("MAMUTE_ZSPLIT", str(zsplit))
    monkeypatch.setenv("MAMUTE_ADJ_ZSPLIT", str(zsplit))
    np.testing.assert_array_equal(gpu_model(ctx, w), ref)
    J, g = gpu_gradient(ctx, w, dobs, n_snapshots=3)
    assert J == Jr
    np.testing.assert_array_equal(g, gr)


def test_host_entry_point_matches_device(ctx):
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=5)
    dev_out = gpu_model(ctx, w)
    host_out = np.zeros_like(dev_out, dtype=np.float32)
    ctx.model_host(mamute.grid_of(w), np.ascontiguousarray(w.vel), np.ascontiguousarray(w.rho),
                   w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, host_out)
    np.testing.assert_array_equal(host_out, dev_out)


def test_pseudo_hessian_matches_oracle(ctx, oracle):
    w = synth.small_case(seed=6, nt=40)
    ph = torch.zeros(w.vel.shape, device="cuda:0")
    gpu_model(ctx, w, phess=ph)
    _, ref = oracle.model(ogrid(oracle, w), w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                          rho=w.rho, phess=True)
    assert rel(ph.cpu().numpy(), ref) <= 1e-4


def _grad_case(density, seed=7, nt=50):
    return synth.small_case(seed=seed, nx=26, ny=22, nz=20, border=6, nt=nt, density=density,
                            n_src=2, n_rec=9)


@pytest.mark.parametrize("density", [False, True])
def test_gradient_matches_oracle(ctx, oracle, density):
    w = _grad_case(density)
    og = ogrid(oracle, w)
    rng = np.random.default_rng(3)
    vtrue = (w.vel * (1 + 0.05 * rng.standard_normal(w.vel.shape))).astype(np.float32)
    dobs = oracle.model(og, vtrue, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    dobs32 = dobs.astype(np.float32)
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs32,
                             rho=w.rho)
    J, g = gpu_gradient(ctx, w, dobs32, n_snapshots=5)
    assert np.isfinite(g).all()
    assert cosine(g, gr) >= GRAD_COS
    assert abs(J - Jr) <= 1e-4 * Jr
    assert rel(g, gr) <= 1e-3


def test_gradient_bitwise_identical_across_snapshot_modes(ctx):
    w = _grad_case(True, seed=8, nt=33)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt), np.float32)
    J0, g0 = gpu_gradient(ctx, w, dobs, n_snapshots=-1)
    for ns in (1, 2, 5, 32, 0):
        J, g = gpu_gradient(ctx, w, dobs, n_snapshots=ns)
        assert J == J0
        np.testing.assert_array_equal(g, g0)


def test_pseudo_hessian_with_all_terms_storage(ctx, oracle):
    """The pseudo-Hessian is accumulated in the all-terms forward sweep too:
    with every imaging term kept, the gradient is bitwise the one without
    the pseudo-Hessian, and P matches the revolve-mode P bitwise and the
    oracle to 1e-4."""
    w = _grad_case(True, seed=14, nt=31)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt), np.float32)
    J0, g0 = gpu_gradient(ctx, w, dobs, n_snapshots=-1)
    ph_all = torch.zeros(w.vel.shape, device="cuda:0")
    J1, g1 = gpu_gradient(ctx, w, dobs, n_snapshots=-1, phess=ph_all)
    ph_rev = torch.zeros(w.vel.shape, device="cuda:0")
    J2, g2 = gpu_gradient(ctx, w, dobs, n_snapshots=3, phess=ph_rev)
    assert J1 == J0 and J2 == J0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(g2, g0)
    np.testing.assert_array_equal(ph_all.cpu().numpy(), ph_rev.cpu().numpy())
    _, ref = oracle.model(ogrid(oracle, w), w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                          rho=w.rho, phess=True)
    assert rel(ph_all.cpu().numpy(), ref) <= 1e-4


def test_automatic_storage_keeps_every_term_when_it_fits(ctx):
    """n_snapshots = 0 on a small grid keeps every imaging term: one forward
    and one adjoint launch per step, and the all-states result."""
    import ctypes
    from paper_2502_12350_gb300 import mamute
    lib = mamute.load()
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    w = _grad_case(True, seed=12, nt=29)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt), np.float32)
    J0, g0 = gpu_gradient(ctx, w, dobs, n_snapshots=-1)
    lib.mamute_ctx_set_timing(ctx._h, 1)
    try:
        J, g = gpu_gradient(ctx, w, dobs, n_snapshots=0)
        sl = ctypes.c_longlong()
        lib.mamute_ctx_last_timing(ctx._h, None, ctypes.byref(sl), None)
        Jr, gr = gpu_gradient(ctx, w, dobs, n_snapshots=3)
        slr = ctypes.c_longlong()
        lib.mamute_ctx_last_timing(ctx._h, None, ctypes.byref(slr), None)
    finally:
        lib.mamute_ctx_set_timing(ctx._h, 0)
    assert sl.value == 2 * w.nt
    assert slr.value > 2 * w.nt  # revolve with 3 slots recomputes
    assert J == J0 and Jr == J0
    np.testing.assert_array_equal(g, g0)
    np.testing.assert_array_equal(gr, g0)


def test_adjoint_is_transpose_applied_to_data(ctx, oracle):
    """mamute_adjoint(d_res) equals the oracle gradient whose residual is d_res."""
    from paper_2502_12350_gb300 import mamute
    w = _grad_case(True, seed=9, nt=40)
    og = ogrid(oracle, w)
    rng = np.random.default_rng(4)
    dres = rng.standard_normal((int(w.rec_offset[-1]), w.nt)).astype(np.float32)
    d = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    _, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                            d - dres.astype(np.float64), rho=w.rho)
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(w.vel).to(dev)
    rho = torch.from_numpy(w.rho).to(dev)
    grad = torch.zeros_like(vel)
    ctx.adjoint(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                torch.from_numpy(dres).to(dev), grad, n_snapshots=3)
    assert cosine(grad.cpu().numpy(), gr) >= GRAD_COS


def test_zero_top_planes(ctx):
    w = _grad_case(False, seed=10, nt=30)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt), np.float32)
    _, g0 = gpu_gradient(ctx, w, dobs, n_snapshots=4)
    _, g3 = gpu_gradient(ctx, w, dobs, n_snapshots=4, zero_top_planes=3)
    assert np.all(g3[:3] == 0)
    np.testing.assert_array_equal(g3[3:], g0[3:])


def test_errors_are_reported(ctx):
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=12)
    w.vel = w.vel * 3.0  # c dt / h above 0.4529
    with pytest.raises(mamute.MamuteError) as e:
        gpu_model(ctx, w)
    assert e.value.code == mamute.ECFL
    w = synth.small_case(seed=12)
    w.rec_xyz = w.rec_xyz.copy()
    w.rec_xyz[0, 0] = -50.0
    with pytest.raises(mamute.MamuteError) as e:
        gpu_model(ctx, w)
    assert e.value.code == mamute.EINVAL
    w = synth.small_case(seed=12)
    w.aperture = np.array([[1, 10, 0, 10]] * w.n_src, np.int32)
    with pytest.raises(mamute.MamuteError) as e:
        gpu_model(ctx, w)
    assert e.value.code == mamute.EINVAL


def _aperture_case(density, nt=50, seed=30):
    """Several shots, each confined to its own aperture window of a shared
    model (the batched layout): x starts on multiples of 4, ragged sizes."""
    w = synth.small_case(seed=seed, nx=52, ny=44, nz=16, border=5, nt=nt, density=density,
                         n_src=4, n_rec=6, fpeak=30.0)
    rng = np.random.default_rng(seed)
    aps, srcs, recs = [], [], []
    for s in range(4):
        x0 = 4 * int(rng.integers(0, 6))
        x1 = min(w.nx, x0 + int(rng.integers(17, 31)))
        y0 = int(rng.integers(0, 15))
        y1 = min(w.ny, y0 + int(rng.integers(15, 29)))
        aps.append((x0, x1, y0, y1))
        srcs.append(((x0 + x1) // 2, (y0 + y1) // 2, int(rng.integers(2, w.nz - 2))))
        for r in range(6):
            recs.append((int(rng.integers(x0, x1)), int(rng.integers(y0, y1)),
                         int(rng.integers(0, w.nz))))
    w.aperture = np.array(aps, np.int32)
    w.src_xyz = (np.array(srcs) * w.h).astype(np.float32)
    w.rec_xyz = (np.array(recs) * w.h).astype(np.float32)
    w.rec_offset = np.arange(5, dtype=np.int32) * 6
    return w


@pytest.mark.parametrize("density", [False, True])
def test_aperture_batch_model_and_gradient(ctx, oracle, density):
    w = _aperture_case(density)
    og = ogrid(oracle, w)
    got = gpu_model(ctx, w)
    ref = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       aperture=w.aperture)
    assert rel(got, ref) <= SEIS_TOL_64
    rng = np.random.default_rng(5)
    dobs = oracle.model(og, w.vel * (1 + 0.05 * rng.standard_normal(w.vel.shape)), w.src_xyz,
                        w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                        aperture=w.aperture).astype(np.float32)
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                             rho=w.rho, aperture=w.aperture)
    J, g = gpu_gradient(ctx, w, dobs, n_snapshots=4)
    assert cosine(g, gr) >= GRAD_COS
    assert rel(g, gr) <= 1e-3
    assert abs(J - Jr) <= 1e-4 * Jr
    # Every stored term covers the window cells inside the model (the
    # window's own sponge included, as in the recomputing mode), so keeping
    # every term gives the revolve result bit for bit.
    Ja, ga = gpu_gradient(ctx, w, dobs, n_snapshots=-1)
    assert Ja == J
    np.testing.assert_array_equal(ga, g)

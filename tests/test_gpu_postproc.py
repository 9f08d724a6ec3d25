"""Parity of the gradient smoothing filters and the data time resampling
(CUDA path through the C ABI) with the oracle, alone and inside
mamute_model / mamute_gradient."""
import numpy as np
import pytest

from oracle import postproc
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


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def cosine(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return a @ b / (np.linalg.norm(a) * np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(18, 20, 24), (20, 36, 70), (5, 3, 130)])
@pytest.mark.parametrize("mode", [1, 2])
def test_smooth_matches_oracle(ctx, shape, mode):
    rng = np.random.default_rng(sum(shape) + mode)
    g = rng.standard_normal(shape).astype(np.float32)
    h = 12.5
    lengths = (2 * h, 3 * h, 1.5 * h)
    ref = postproc.smooth(g, h, mode, lengths)
    dev = torch.device("cuda:0")
    gi = torch.from_numpy(g).to(dev)
    out = torch.full_like(gi, float("nan"))
    ctx.smooth(h, mode, gi, out, lengths=lengths)
    assert rel(out.cpu().numpy(), ref) <= 1e-5
    ctx.smooth(h, mode, gi, gi, lengths=lengths)  # in place
    np.testing.assert_array_equal(gi.cpu().numpy(), out.cpu().numpy())


@pytest.mark.parametrize("case", [(301, 1e-3, 80, 3.7e-3), (120, 4e-3, 470, 1e-3),
                                  (64, 2e-3, 64, 2e-3)])
@pytest.mark.parametrize("mode", [1, 2])
def test_resample_matches_oracle(ctx, case, mode):
    nt_in, dt_in, nt_out, dt_out = case
    # the library takes FP32 steps; the oracle gets the same values, so both
    # take the nearest-sample decisions on the same numbers (in FP64)
    dt_in, dt_out = float(np.float32(dt_in)), float(np.float32(dt_out))
    rng = np.random.default_rng(nt_in + mode)
    x = rng.standard_normal((37, nt_in)).astype(np.float32)
    name = {1: "nearest", 2: "sinc"}[mode]
    ref = postproc.resample(x, dt_in, nt_out, dt_out, name)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    y = torch.full((37, nt_out), float("nan"), device=dev)
    ctx.resample(xt, dt_in, nt_out, dt_out, mode, y)
    if mode == 1:
        np.testing.assert_array_equal(y.cpu().numpy(), ref.astype(np.float32))
    else:
        assert rel(y.cpu().numpy(), ref) <= 1e-5
    # the transpose
    r = rng.standard_normal((37, nt_out)).astype(np.float32)
    refT = postproc.resample(r, dt_in, None, dt_out, name, adjoint=True, nt_in=nt_in)
    yt = torch.full((37, nt_in), float("nan"), device=dev)
    ctx.resample(torch.from_numpy(r).to(dev), dt_in, nt_out, dt_out, mode, yt, adjoint=True)
    # (nearest: several outputs may share a sample, whose transpose sums them in FP32)
    assert rel(yt.cpu().numpy(), refT) <= (1e-6 if mode == 1 else 1e-5)
    if mode == 1:  # the index decisions themselves: the same support exactly
        np.testing.assert_array_equal(yt.cpu().numpy() != 0, refT != 0)


def _case():
    return synth.small_case(seed=101, nx=26, ny=22, nz=20, border=6, nt=64, density=True,
                            n_src=2, n_rec=9)


def _dev(w):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(w.vel).to(dev), torch.from_numpy(w.rho).to(dev))


@pytest.mark.parametrize("mode", [1, 2])
def test_gradient_smoothing_matches_oracle(ctx, oracle, mode):
    from paper_2502_12350_gb300 import mamute
    w = _case()
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    rng = np.random.default_rng(5)
    dobs = oracle.model(og, w.vel * (1 + 0.05 * rng.standard_normal(w.vel.shape)), w.src_xyz,
                        w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho).astype(np.float32)
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                             rho=w.rho)
    lengths = (2.5 * w.h, 2 * w.h, 1.5 * w.h)
    ref = postproc.smooth(gr, w.h, mode, lengths)
    ref[:3] = 0.0  # ZeroesNearSurface after the filter
    vel, rho = _dev(w)
    grad = torch.full_like(vel, float("nan"))
    J = ctx.gradient(mamute.grid_of(w), vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                     torch.from_numpy(dobs).to(vel.device), grad, n_snapshots=4,
                     smooth_mode=mode, smooth_len=lengths, zero_top_planes=3)
    g = grad.cpu().numpy()
    assert np.all(g[:3] == 0)
    assert cosine(g, ref) >= 0.9999
    assert abs(J - Jr) <= 1e-4 * Jr


@pytest.mark.parametrize("mode", [1, 2])
def test_model_and_gradient_on_a_data_time_axis(ctx, oracle, mode):
    """Data at dt_data = 2.5 dt (nt_data samples): modelled traces are
    resampled to the data axis, J = 1/2 |K d - d_obs|^2 and the adjoint source
    is K^T (K d - d_obs)."""
    from paper_2502_12350_gb300 import mamute
    w = _case()
    name = {1: "nearest", 2: "sinc"}[mode]
    dt_data, nt_data = float(np.float32(2.5 * w.dt)), 25
    w.dt = float(np.float32(w.dt))
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    d = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    Kd = postproc.resample(d, w.dt, nt_data, dt_data, name)
    vel, rho = _dev(w)
    n_rec = int(w.rec_offset[-1])
    seis = torch.full((n_rec, nt_data), float("nan"), device=vel.device)
    g = mamute.grid_of(w)
    ax = dict(time_interp=mode, nt_data=nt_data, dt_data=dt_data)
    ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis, **ax)
    assert rel(seis.cpu().numpy(), Kd) <= 1e-4
    rng = np.random.default_rng(6)
    dobs = (Kd * (1 + 0.1 * rng.standard_normal(Kd.shape))).astype(np.float32)
    res = Kd - dobs
    Jr = 0.5 * np.sum(res ** 2)
    adj_src = postproc.resample(res, w.dt, None, dt_data, name, adjoint=True, nt_in=w.nt)
    _, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                            d - adj_src, rho=w.rho)
    grad = torch.full_like(vel, float("nan"))
    J = ctx.gradient(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                     torch.from_numpy(dobs).to(vel.device), grad, n_snapshots=-1, **ax)
    assert abs(J - Jr) <= 1e-4 * Jr
    assert cosine(grad.cpu().numpy(), gr) >= 0.9999
    # the host entry point on the data axis (copies after the resampling)
    host = np.zeros((n_rec, nt_data), np.float32)
    ctx.model_host(g, np.ascontiguousarray(w.vel), np.ascontiguousarray(w.rho), w.src_xyz,
                   w.wavelet, w.rec_offset, w.rec_xyz, host, **ax)
    np.testing.assert_array_equal(host, seis.cpu().numpy())


def test_cached_tables_follow_the_call(ctx):
    """The transform tables and the resampling matrix are kept between calls
    with the same sizes and parameters: alternating parameters must give,
    call for call, what a fresh context gives."""
    from paper_2502_12350_gb300 import mamute
    rng = np.random.default_rng(61)
    g = torch.from_numpy(rng.standard_normal((12, 14, 20)).astype(np.float32)).cuda()
    x = torch.from_numpy(rng.standard_normal((7, 90)).astype(np.float32)).cuda()
    calls = [("smooth", 1, (20.0, 30.0, 10.0)), ("smooth", 2, (20.0, 30.0, 10.0)),
             ("smooth", 1, (40.0, 30.0, 10.0)), ("smooth", 1, (20.0, 30.0, 10.0)),
             ("resample", mamute.INTERP_SINC, 0), ("resample", mamute.INTERP_NEAREST, 0),
             ("resample", mamute.INTERP_SINC, 1), ("resample", mamute.INTERP_SINC, 0)]

    def run(c, call):
        if call[0] == "smooth":
            out = torch.empty_like(g)
            c.smooth(10.0, call[1], g, out, lengths=call[2])
        elif call[2] == 0:
            out = torch.empty((7, 40), device="cuda:0")
            c.resample(x, 1e-3, 40, 2.2e-3, call[1], out)
        else:
            out = torch.empty((7, 90), device="cuda:0")
            c.resample(x[:, :40].contiguous(), 1e-3, 40, 2.2e-3, call[1], out, adjoint=True)
        return out.cpu().numpy()

    for call in calls:
        got = run(ctx, call)
        fresh = mamute.Context(0)
        try:
            want = run(fresh, call)
        finally:
            fresh.close()
        np.testing.assert_array_equal(got, want, err_msg=str(call))

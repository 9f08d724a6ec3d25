"""The two-level forward kernel (two time steps per pass, tiles exchanging
u^{n+1} halos through L2) against the one-step kernel and the oracle.

Every point goes through the same operations in the same order, so the
seismograms must be bitwise those of the one-step path; the launch count
shows which path ran."""
import ctypes

import numpy as np
import pytest

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
    lib = mamute.load()
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.mamute_ctx_set_timing(c._h, 1)
    yield c
    lib.mamute_ctx_set_timing(c._h, 0)
    c.close()


def _model(ctx, w, xi=0):
    from paper_2502_12350_gb300 import mamute
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.vel)).to(dev)
    rho = None if w.rho is None else torch.from_numpy(np.ascontiguousarray(w.rho)).to(dev)
    seis = torch.full((int(w.rec_offset[-1]), w.nt), float("nan"), device=dev)
    ctx.model(mamute.grid_of(w, xyz_interp=xi), vel, rho, w.src_xyz, w.wavelet, w.rec_offset,
              w.rec_xyz, seis, time_blocking=2)
    sl = ctypes.c_longlong()
    ctx.lib.mamute_ctx_last_timing(ctx._h, None, ctypes.byref(sl), None)
    return seis.cpu().numpy(), sl.value


CASES = [
    dict(seed=120, nx=40, ny=36, nz=28, border=8, nt=64, density=True, n_src=1, n_rec=12),
    dict(seed=121, nx=70, ny=45, nz=21, border=6, nt=51, density=False, n_src=1, n_rec=9),
    dict(seed=122, nx=150, ny=97, nz=17, border=5, nt=40, density=True, n_src=1, n_rec=20),
]


@pytest.mark.parametrize("case", CASES)
def test_pairs_bitwise_equal_one_step_and_match_oracle(ctx, oracle, monkeypatch, case):
    w = synth.small_case(**case)
    two, launches = _model(ctx, w)
    assert launches == (w.nt + 1) // 2  # two steps per launch (+1 for an odd count)
    monkeypatch.setenv("MAMUTE_PAIRS", "0")
    one, launches1 = _model(ctx, w)
    assert launches1 == w.nt
    np.testing.assert_array_equal(two, one)
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    ref = oracle.model(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    assert np.linalg.norm(two - ref) / np.linalg.norm(ref) <= 1e-4


def test_pairs_with_offgrid_points_and_host_copies(ctx, monkeypatch):
    from paper_2502_12350_gb300 import mamute
    w = synth.small_case(seed=123, nx=48, ny=40, nz=22, border=6, nt=58, n_src=1, n_rec=15)
    rng = np.random.default_rng(3)
    w.src_xyz = (w.src_xyz + 0.4 * w.h).astype(np.float32)
    w.rec_xyz = np.clip(w.rec_xyz + rng.uniform(0.1, 0.9, w.rec_xyz.shape) * w.h, 0,
                        (np.array([w.nx, w.ny, w.nz]) - 1) * w.h - 1e-3).astype(np.float32)
    two, _ = _model(ctx, w, xi=1)
    host = np.zeros_like(two)
    ctx.model_host(mamute.grid_of(w, xyz_interp=1), np.ascontiguousarray(w.vel),
                   np.ascontiguousarray(w.rho), w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                   host, time_blocking=2)
    np.testing.assert_array_equal(host, two)
    monkeypatch.setenv("MAMUTE_PAIRS", "0")
    one, _ = _model(ctx, w, xi=1)
    np.testing.assert_array_equal(two, one)

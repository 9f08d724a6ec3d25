"""The allocation-free misfit entry point, for callers that cannot allocate
device memory (a framework allocator already holding the device's memory, or
a loop that must not pay for cudaMalloc's device-wide synchronisation).

It is called through the C ABI and compared with the misfit that
mamute_gradient returns for the same modelled and observed data and with an
FP64 host sum of the same arrays, on two calls in a row (the second call
reuses the fixed scratch the first one left behind).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2502_12350_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, mamute
    build.build()
    so = mamute.load()
    so.mamute_misfit_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    so.mamute_misfit_noalloc.restype = ctypes.c_int
    return mamute, so


def test_noalloc_misfit_matches_gradient_misfit(lib):
    mamute, so = lib
    dev = torch.device("cuda:0")
    ctx = mamute.Context(0)
    try:
        w = synth.small_case(seed=41, nx=30, ny=26, nz=20, border=6, nt=70, n_src=3, n_rec=11)
        g = mamute.grid_of(w)
        vel = torch.from_numpy(w.vel).to(dev)
        rho = torch.from_numpy(w.rho).to(dev)
        n_rec = int(w.rec_offset[-1])
        d = torch.empty((n_rec, w.nt), device=dev)
        ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, d)
        stream = torch.cuda.current_stream(dev).cuda_stream
        for trial in range(2):
            rng = np.random.default_rng(100 + trial)
            dobs = (d.cpu().numpy() * (1.0 + 0.1 * (trial + 1)) +
                    1e-3 * np.abs(d.cpu().numpy()).max() *
                    rng.standard_normal(d.shape)).astype(np.float32)
            dobs_t = torch.from_numpy(dobs).to(dev)
            grad = torch.empty_like(vel)
            J_ref = ctx.gradient(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                                 dobs_t, grad, n_snapshots=4)
            J = ctypes.c_double(-1.0)
            rc = so.mamute_misfit_noalloc(ctypes.c_void_p(d.data_ptr()),
                                          ctypes.c_void_p(dobs_t.data_ptr()),
                                          d.numel(), ctypes.c_void_p(stream), ctypes.byref(J))
            assert rc == mamute.OK
            assert J.value > 0
            # the same formula in the same summation order as the gradient's
            assert abs(J.value - J_ref) <= 1e-9 * J_ref, (trial, J.value, J_ref)
            assert J.value == J_ref, (trial, J.value, J_ref)
            # and the definition itself, summed on the host in FP64 from the
            # FP32 residuals of the same two arrays
            r32 = d.cpu().numpy() - dobs  # FP32 residual, as on the device
            J_host = 0.5 * float(np.sum(r32.astype(np.float64) ** 2))
            assert abs(J.value - J_host) <= 1e-12 * J_host, (trial, J.value, J_host)
    finally:
        ctx.close()


def test_noalloc_misfit_rejects_oversize_and_nulls(lib):
    mamute, so = lib
    dev = torch.device("cuda:0")
    a = torch.zeros(8, device=dev)
    J = ctypes.c_double(-1.0)
    big = 16384 * 16384 + 1
    assert so.mamute_misfit_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                    big, None, ctypes.byref(J)) == mamute.EINVAL
    assert so.mamute_misfit_noalloc(None, None, 8, None, ctypes.byref(J)) == mamute.EINVAL
    assert J.value == -1.0
    assert so.mamute_misfit_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                    8, None, ctypes.byref(J)) == mamute.OK
    assert J.value == 0.0

"""The autograd binding: its backward equals the oracle gradient and a
finite-difference check of the FP32 forward along a smooth perturbation."""
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
    yield c
    c.close()


def _setup(ctx, density, seed=21, nt=60):
    from paper_2502_12350_gb300 import autograd, mamute
    w = synth.small_case(seed=seed, nx=28, ny=24, nz=20, border=6, nt=nt, density=density,
                         n_src=2, n_rec=12)
    acq = autograd.Acquisition(mamute.grid_of(w), w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                               n_snapshots=6)
    return w, acq


@pytest.mark.parametrize("density", [False, True])
def test_backward_matches_oracle_gradient(ctx, oracle, density):
    from paper_2502_12350_gb300 import autograd
    w, acq = _setup(ctx, density)
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(0)
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    dobs = oracle.model(og, w.vel * (1 + 0.04 * rng.standard_normal(w.vel.shape)), w.src_xyz,
                        w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho).astype(np.float32)
    vel = torch.from_numpy(w.vel).to(dev).requires_grad_(True)
    rho = None if w.rho is None else torch.from_numpy(w.rho).to(dev)
    seis = autograd.propagate(vel, acq, ctx, rho)
    loss = 0.5 * ((seis.double() - torch.from_numpy(dobs).to(dev).double()) ** 2).sum()
    loss.backward()
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                             rho=w.rho)
    g = vel.grad.cpu().numpy().astype(np.float64).ravel()
    cos = g @ gr.ravel() / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert cos >= 0.9999
    assert abs(loss.item() - Jr) <= 1e-4 * Jr


def test_backward_matches_finite_differences(ctx):
    """Central differences of the FP32 forward along a smooth, large-scale
    perturbation that vanishes on the outer model layer."""
    from paper_2502_12350_gb300 import autograd
    w, acq = _setup(ctx, False, seed=22, nt=80)
    dev = torch.device("cuda:0")
    vel0 = torch.from_numpy(w.vel).to(dev)
    nz, ny, nx = w.vel.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bump = np.exp(-(((x - nx / 2) / 5) ** 2 + ((y - ny / 2) / 5) ** 2 + ((z - nz / 2) / 4) ** 2))
    bump[[0, -1], :, :] = 0
    bump[:, [0, -1], :] = 0
    bump[:, :, [0, -1]] = 0
    dc = torch.from_numpy(bump.astype(np.float32)).to(dev)
    rng = np.random.default_rng(1)
    wr = torch.from_numpy(rng.standard_normal((acq.n_rec, w.nt)).astype(np.float32)).to(dev)
    vel = vel0.clone().requires_grad_(True)
    (autograd.propagate(vel, acq, ctx) * wr).double().sum().backward()
    pred = (vel.grad.double() * dc.double()).sum().item()
    eps = 20.0  # m/s: large enough to stand out of FP32 rounding, small for O(eps^2)
    with torch.no_grad():
        fp = (autograd.propagate(vel0 + eps * dc, acq, ctx).double() * wr.double()).sum().item()
        fm = (autograd.propagate(vel0 - eps * dc, acq, ctx).double() * wr.double()).sum().item()
    fd = (fp - fm) / (2 * eps)
    assert abs(fd - pred) <= 2e-3 * abs(pred), (fd, pred)

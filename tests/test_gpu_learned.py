"""What the learned preconditioner gains over the method without it.

The network is trained (on the GPU, by the library's kernels) on exact
Gauss-Newton diagonals of small seeded models; on held-out models its
prediction of log H must be clearly closer to the exact diagonal than the
pseudo-Hessian, both compared up to a constant factor (the
pseudo-Hessian preconditioner is what the method uses without the network).
A short inversion then checks that both preconditioned L-BFGS runs reduce
the misfit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, cnn, learned, mamute, synth
    build.build()
    ctx = mamute.Context(0)

    def wl(mid):
        return synth.fwi_small(model_id=mid, nt=300, nx=40, ny=40, nz=24, border=10)

    net = cnn.Net(ctx, seed=1)
    train = learned.dataset(ctx, net, wl, list(range(5000, 5016)), seed=1)
    held = learned.dataset(ctx, net, wl, list(range(5380, 5384)), seed=2, set_offset=False)
    yield ctx, net, learned, wl, train, held
    ctx.close()


def test_network_beats_pseudo_hessian_on_heldout_models(setup):
    ctx, net, learned, wl, train, held = setup
    before = learned.log_errors(net, held)
    hist = learned.train(net, train, epochs=60, lr=3e-3)
    assert hist[-1] < 0.7 * hist[0]
    after = learned.log_errors(net, held)
    net_err = np.mean([e[0] for e in after])
    p_err = np.mean([e[1] for e in after])
    assert np.mean([e[0] for e in before]) > net_err
    assert net_err < 0.8 * p_err, (net_err, p_err)


def test_preconditioned_fwi_reduces_misfit(setup):
    from paper_2502_12350_gb300 import fwi, mamute
    ctx, net, learned, wl, train, held = setup
    w = wl(5390)
    dev = torch.device("cuda:0")
    dobs = torch.empty((int(w.rec_offset[-1]), w.nt), device=dev)
    ctx.model(mamute.grid_of(w), torch.from_numpy(w.vel).to(dev), None, w.src_xyz, w.wavelet,
              w.rec_offset, w.rec_xyz, dobs)
    for kind in ("pseudo", "learned"):
        prob = fwi.Problem(ctx, w, dobs, 1400.0, 5000.0)
        res = fwi.run(prob, w.vel_init.astype(np.float64), 3, precond=kind, net=net)
        assert res.history[-1][1] < 0.97 * res.history[0][1], (kind, res.history)

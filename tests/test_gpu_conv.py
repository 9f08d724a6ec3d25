"""The network kernels against the FP64 conv3d oracle on BF16-exact inputs:
forward convolution, input gradient (flipped weights), weight and bias
gradients, the full network loss and gradients, and training progress."""
import numpy as np
import pytest

from oracle import conv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_12350_gb300 import build, cnn, mamute
    build.build()
    ctx = mamute.Context(0)
    yield ctx, cnn
    ctx.close()


def _bf16_bits(a):
    """FP64 values that are exact BF16 -> int16 bit patterns (channels last)."""
    f = np.asarray(a, np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def _from_bits(t):
    return (t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32)


def _rand_act(rng, D, H, W, ch):
    x = np.zeros((D, H, W, 16), np.float32)
    x[..., :ch] = rng.standard_normal((D, H, W, ch))
    return conv.bf16_round(x)


# ragged tiles in every axis; two x segments (W > 198); many row blocks with
# z chunks of 3 planes per persistent CTA item
SHAPES = [(3, 8, 16), (5, 11, 21), (2, 9, 33), (2, 3, 205), (8, 200, 198)]


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_forward_and_input_gradient(net_mod, shape):
    ctx, cnn = net_mod
    rng = np.random.default_rng(sum(shape))
    D, H, W = shape
    x = _rand_act(rng, D, H, W, 16)
    w = conv.bf16_round((0.2 * rng.standard_normal((27, 16, 16))).astype(np.float32))
    b = rng.standard_normal(16).astype(np.float32)
    dev = torch.device("cuda:0")
    net = cnn.Net(ctx, weights=([w.astype(np.float32)] * 4, [b] * 4))
    xt = torch.from_numpy(_bf16_bits(x)).to(dev)
    y32 = torch.zeros((D, H, W, 16), device=dev)
    lib = net.lib
    net._check(lib.mamute_conv3d(ctx._h, D, H, W, cnn._p(xt), cnn._p(net.wf[0]), cnn._p(net.b[0]),
                                 0, None, cnn._p(y32), None))
    wo = cnn.to_oracle_layout(w)
    ref = conv.forward(np.moveaxis(x, -1, 0), wo, b)
    got = np.moveaxis(y32.cpu().numpy(), -1, 0)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # input gradient with the flipped weight set, masked by a random ReLU pattern
    gy = _rand_act(rng, D, H, W, 16)
    mask = _rand_act(rng, D, H, W, 16)
    g16 = torch.zeros((D, H, W, 16), dtype=torch.int16, device=dev)
    g32 = torch.zeros((D, H, W, 16), device=dev)
    gyt = torch.from_numpy(_bf16_bits(gy)).to(dev)  # held: the call gets raw pointers
    mt = torch.from_numpy(_bf16_bits(mask)).to(dev)
    net._check(lib.mamute_conv3d(ctx._h, D, H, W, cnn._p(gyt), cnn._p(net.wb[0]), None, 0,
                                 cnn._p(mt), cnn._p(g32), cnn._p(g16)))
    refg = conv.backward_input(np.moveaxis(gy, -1, 0), wo) * (np.moveaxis(mask, -1, 0) > 0)
    gotg = np.moveaxis(g32.cpu().numpy(), -1, 0)
    assert np.abs(gotg - refg).max() <= 1e-5 * np.abs(refg).max()
    np.testing.assert_array_equal(_from_bits(g16), conv.bf16_round(g32.cpu().numpy()).astype(np.float32))


@pytest.mark.parametrize("shape", SHAPES)
def test_weight_gradient(net_mod, shape):
    ctx, cnn = net_mod
    rng = np.random.default_rng(7 + sum(shape))
    D, H, W = shape
    x = _rand_act(rng, D, H, W, 16)
    gy = _rand_act(rng, D, H, W, 16)
    dev = torch.device("cuda:0")
    net = cnn.Net(ctx)
    gw = torch.zeros((27, 16, 16), device=dev)
    gb = torch.zeros(16, device=dev)
    xt = torch.from_numpy(_bf16_bits(x)).to(dev)  # held: the call gets raw pointers
    gyt = torch.from_numpy(_bf16_bits(gy)).to(dev)
    net._check(net.lib.mamute_conv3d_wgrad(ctx._h, D, H, W, cnn._p(xt), cnn._p(gyt), cnn._p(gw),
                                           cnn._p(gb)))
    rw, rb = conv.backward_weight(np.moveaxis(x, -1, 0), np.moveaxis(gy, -1, 0))
    got = cnn.to_oracle_layout(gw.cpu().numpy())
    assert np.abs(got - rw).max() <= 1e-5 * np.abs(rw).max()
    assert np.abs(gb.cpu().numpy() - rb).max() <= 1e-5 * np.abs(rb).max()


def test_network_loss_and_gradients(net_mod):
    """The full network (BF16 activations on both sides) against the oracle;
    the GPU also stores intermediate gradients in BF16, so weights agree to
    a cosine of 0.999."""
    ctx, cnn = net_mod
    rng = np.random.default_rng(11)
    D, H, W = 6, 12, 20
    ws, bs = cnn.init_weights(3)
    ws = [conv.bf16_round(w).astype(np.float32) for w in ws]
    bs = [0.05 * rng.standard_normal(16).astype(np.float32) for _ in range(4)]
    x = _rand_act(rng, D, H, W, 2)
    t = rng.standard_normal((D, H, W)).astype(np.float32)
    dev = torch.device("cuda:0")
    net = cnn.Net(ctx, weights=(ws, bs))
    loss = net.loss_and_grads(torch.from_numpy(_bf16_bits(x)).to(dev), torch.from_numpy(t).to(dev))
    onet = conv.Net([cnn.to_oracle_layout(w)[:cnn.CHANNELS[l + 1], :cnn.CHANNELS[l]]
                     for l, w in enumerate(ws)],
                    [b[:cnn.CHANNELS[l + 1]] for l, b in enumerate(bs)])
    rl, rgw, rgb = onet.loss_and_grads(np.moveaxis(x, -1, 0)[:2], t)
    assert abs(loss - rl) <= 1e-4 * rl
    for l in range(4):
        g = cnn.to_oracle_layout(net.gw[l].cpu().numpy())[:cnn.CHANNELS[l + 1], :cnn.CHANNELS[l]]
        cos = np.sum(g * rgw[l]) / (np.linalg.norm(g) * np.linalg.norm(rgw[l]))
        assert cos >= 0.999, (l, cos)


def test_training_reduces_loss(net_mod):
    ctx, cnn = net_mod
    rng = np.random.default_rng(12)
    D, H, W = 8, 16, 16
    dev = torch.device("cuda:0")
    x = _rand_act(rng, D, H, W, 2)
    # a smooth target the network can represent: a local mix of the inputs
    t = (0.7 * x[..., 0] - 0.4 * x[..., 1]).astype(np.float32)
    net = cnn.Net(ctx, seed=4)
    xt, tt = torch.from_numpy(_bf16_bits(x)).to(dev), torch.from_numpy(t).to(dev)
    losses = [net.train_step(xt, tt, lr=3e-3) for _ in range(150)]
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def test_network_features(net_mod):
    """Input channels and log-ratio target against a float64 restatement:
    channel 0 = (c - v_ref) / v_scale, channel 1 = clipped log(P / Pmax)
    / clip (both rounded to BF16), channels 2..15 zero, target = log(H / P)."""
    ctx, cnn = net_mod
    rng = np.random.default_rng(11)
    D, H, W = 5, 7, 9
    vel = rng.uniform(1500.0, 4500.0, (D, H, W)).astype(np.float32)
    ph = np.exp(rng.uniform(-30.0, 0.0, (D, H, W))).astype(np.float32) * 3.0
    hd = np.exp(rng.uniform(-10.0, 2.0, (D, H, W))).astype(np.float32)
    dev = torch.device("cuda:0")
    net = cnn.Net(ctx, seed=0)
    x16, tgt, pmax = net.features(torch.from_numpy(vel).to(dev), torch.from_numpy(ph).to(dev),
                                  torch.from_numpy(hd).to(dev), 3000.0, 1000.0, 20.0)
    assert pmax == float(ph.max())
    x = _from_bits(x16).astype(np.float64)
    c = (vel.astype(np.float64) - 3000.0) / 1000.0
    lp = np.maximum(np.log(ph.astype(np.float64) / ph.max()), -20.0) / 20.0
    # BF16 keeps 8 significant bits: half an ulp of rounding plus the FP32 log
    np.testing.assert_allclose(x[..., 0], c, rtol=2.0 ** -8, atol=1e-6)
    np.testing.assert_allclose(x[..., 1], lp, rtol=2.0 ** -8, atol=1e-6)
    assert not x[..., 2:].any()
    t = np.log(hd.astype(np.float64) / ph.astype(np.float64))
    np.testing.assert_allclose(tgt.cpu().numpy(), t, rtol=0, atol=1e-4 * np.abs(t).max())

"""Pins of the conv3d oracle: agreement with torch's CPU conv3d in FP64 (a
library routine for the same textbook sum), transposition identities of the
input and weight gradients, finite differences of the network loss, and the
BF16 rounding rule."""
import numpy as np
import pytest

from oracle import conv


def test_bf16_rounding_rule():
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -2.5, 3.3e38, 1e-40],
                    np.float32)
    r = conv.bf16_round(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert r[1] == 1.0
    assert r[2] == 1.0078125
    assert r[0] == 1.0 and r[3] == 1.0078125 and r[4] == -2.5
    # every rounded value has at most 8 significant bits
    for v in r[np.isfinite(r) & (r != 0)]:
        m = np.frexp(v)[0] * 2**8
        assert abs(m - round(m)) < 1e-9


def test_forward_matches_torch_conv3d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = torch.nn.functional.conv3d(torch.from_numpy(x)[None], torch.from_numpy(w),
                                     torch.from_numpy(b), padding=1)[0].numpy()
    np.testing.assert_allclose(conv.forward(x, w, b), ref, rtol=1e-12, atol=1e-12)


def test_adjoint_identities():
    """<conv(x), g> = <x, backward_input(g)> = <w, backward_weight(x, g)>."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    g = rng.standard_normal((2, 4, 5, 6))
    y = conv.forward(x, w)
    lhs = np.sum(y * g)
    assert abs(lhs - np.sum(x * conv.backward_input(g, w))) < 1e-10 * abs(lhs)
    gw, gb = conv.backward_weight(x, g)
    assert abs(lhs - np.sum(w * gw)) < 1e-10 * abs(lhs)
    np.testing.assert_allclose(gb, g.sum(axis=(1, 2, 3)))


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    ch = [2, 16, 16, 16, 1]
    ws = [0.2 * rng.standard_normal((ch[l + 1], ch[l], 3, 3, 3)) for l in range(4)]
    bs = [0.1 * rng.standard_normal(ch[l + 1]) for l in range(4)]
    # weights exactly representable in BF16 so that perturbations stay exact
    ws = [conv.bf16_round(w.astype(np.float32)) for w in ws]
    x = conv.bf16_round(rng.standard_normal((2, 4, 5, 4)).astype(np.float32))
    t = rng.standard_normal((4, 5, 4))
    net = conv.Net(ws, bs, round_activations=False)
    loss, gws, gbs = net.loss_and_grads(x, t)

    def L(wl, bl):
        return conv.Net(wl, bl, round_activations=False).loss_and_grads(x, t)[0]

    eps = 1e-6
    for l in range(4):
        for o in range(min(3, ch[l + 1])):
            bp = [b.copy() for b in bs]
            bp[l][o] += eps
            bm = [b.copy() for b in bs]
            bm[l][o] -= eps
            fd = (L(ws, bp) - L(ws, bm)) / (2 * eps)
            assert abs(fd - gbs[l][o]) <= 1e-6 * max(1.0, abs(fd)), (l, o, fd, gbs[l][o])
        # one weight per layer, perturbed in FP64 (the oracle does not re-round it)
        wp = [w.copy() for w in ws]
        wp[l][0, 0, 1, 1, 1] += eps
        wm = [w.copy() for w in ws]
        wm[l][0, 0, 1, 1, 1] -= eps
        netp = conv.Net(wp, bs, round_activations=False)
        netp.w = wp
        netm = conv.Net(wm, bs, round_activations=False)
        netm.w = wm
        fd = (netp.loss_and_grads(x, t)[0] - netm.loss_and_grads(x, t)[0]) / (2 * eps)
        assert abs(fd - gws[l][0, 0, 1, 1, 1]) <= 1e-6 * max(1.0, abs(fd)), (l, fd)

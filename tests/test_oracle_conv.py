"""Pins of the FP64 network reference (oracle/conv_ref.py) to things other
than itself: brute-force index loops, a delta kernel that must shift the input,
the adjoint identities of a linear map, finite differences of the loss through
the whole residual network, and Adam's closed-form first step."""
import numpy as np
import pytest

from oracle import conv_ref as cr


def _brute_conv(x, w, b, dil=1):
    n, h, wd, ci = x.shape
    co = w.shape[0]
    y = np.zeros((n, h, wd, co))
    for a in range(n):
        for i in range(h):
            for j in range(wd):
                for o in range(co):
                    s = b[o]
                    for t in range(9):
                        dy, dx = t // 3 - 1, t % 3 - 1
                        for c in range(ci):
                            s += w[o, t, c] * x[a, (i + dil * dy) % h, (j + dil * dx) % wd, c]
                    y[a, i, j, o] = s
    return y


@pytest.mark.parametrize("dil", [1, 2, 3])
def test_conv_matches_brute_force_loops(dil):
    g = np.random.default_rng(1)
    x = g.standard_normal((2, 5, 7, 3))
    w = g.standard_normal((4, 9, 3))
    b = g.standard_normal(4)
    np.testing.assert_allclose(cr.conv3x3(x, w, b, dil), _brute_conv(x, w, b, dil), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dil", [1, 2])
@pytest.mark.parametrize("t", range(9))
def test_delta_kernel_shifts_the_input(t, dil):
    g = np.random.default_rng(2)
    x = g.standard_normal((1, 4, 5, 2))
    w = np.zeros((2, 9, 2))
    w[0, t, 0] = w[1, t, 1] = 1.0
    dy, dx = t // 3 - 1, t % 3 - 1
    y = cr.conv3x3(x, w, dil=dil)
    for i in range(4):
        for j in range(5):
            np.testing.assert_array_equal(y[0, i, j], x[0, (i + dil * dy) % 4, (j + dil * dx) % 5])


@pytest.mark.parametrize("dil", [1, 2])
def test_gradients_are_the_adjoints_of_the_convolution(dil):
    g = np.random.default_rng(3)
    x = g.standard_normal((2, 4, 6, 5))
    w = g.standard_normal((3, 9, 5))
    r = g.standard_normal((2, 4, 6, 3))
    lhs = float((cr.conv3x3(x, w, dil=dil) * r).sum())
    # <conv(x; w), r> = <x, dgrad(r; w)> = <w, wgrad(x, r)>
    assert lhs == pytest.approx(float((x * cr.conv3x3_dgrad(r, w, dil)).sum()), rel=1e-12)
    assert lhs == pytest.approx(float((w * cr.conv3x3_wgrad(x, r, dil)).sum()), rel=1e-12)


def _net(seed, h=4, w=8):
    g = np.random.default_rng(seed)
    weights, biases = [], []
    for ci, co in cr.LAYERS:
        weights.append(g.standard_normal((co, 9, ci)) * np.sqrt(2.0 / (9 * ci)))
        biases.append(g.standard_normal(co) * 0.1)
    x = np.zeros((1, h, w, 16))
    x[..., :5] = g.standard_normal((1, h, w, 5))
    target = np.zeros_like(x)
    target[..., :5] = g.standard_normal((1, h, w, 5))
    return x, target, weights, biases


@pytest.mark.parametrize("dil", [(1,) * 6, (1, 2, 3, 2, 1, 1)])
def test_network_gradients_match_finite_differences(dil):
    x, target, weights, biases = _net(4, h=6, w=8)
    loss, gw, gb = cr.net_loss_and_grads(x, target, weights, biases, dil=dil)
    g = np.random.default_rng(5)
    eps = 1e-6
    for _ in range(24):
        l = int(g.integers(0, 6))
        co, ci = cr.LAYERS[l][1], cr.LAYERS[l][0]
        if g.random() < 0.75:
            # weights of real channels only (padding channels carry nothing)
            o = int(g.integers(0, 5 if l == 5 else co))
            c = int(g.integers(0, 5 if l == 0 else ci))
            t = int(g.integers(0, 9))
            wp = [v.copy() for v in weights]
            wm = [v.copy() for v in weights]
            wp[l][o, t, c] += eps
            wm[l][o, t, c] -= eps
            fd = (cr.net_loss_and_grads(x, target, wp, biases, dil=dil)[0]
                  - cr.net_loss_and_grads(x, target, wm, biases, dil=dil)[0]) / (2 * eps)
            assert gw[l][o, t, c] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        else:
            o = int(g.integers(0, 5 if l == 5 else co))
            bp = [v.copy() for v in biases]
            bm = [v.copy() for v in biases]
            bp[l][o] += eps
            bm[l][o] -= eps
            fd = (cr.net_loss_and_grads(x, target, weights, bp, dil=dil)[0]
                  - cr.net_loss_and_grads(x, target, weights, bm, dil=dil)[0]) / (2 * eps)
            assert gb[l][o] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    assert loss > 0


def test_two_hop_gradients_match_finite_differences():
    """The unrolled two-hop loss (the second hop from the network's own first
    hop) against central differences of itself, weights and biases of every
    layer, with dilated layers."""
    dil = (1, 2, 1, 2, 1, 1)
    x, t1, weights, biases = _net(8, h=6, w=8)
    t2 = np.zeros_like(x)
    t2[..., :5] = np.random.default_rng(9).standard_normal(x[..., :5].shape)
    loss, gw, gb = cr.net_two_hop_loss_and_grads(x, t1, t2, weights, biases, dil=dil)
    g = np.random.default_rng(10)
    eps = 1e-6
    f = lambda w_, b_: cr.net_two_hop_loss_and_grads(x, t1, t2, w_, b_, dil=dil)[0]
    for _ in range(16):
        l = int(g.integers(0, 6))
        co, ci = cr.LAYERS[l][1], cr.LAYERS[l][0]
        o = int(g.integers(0, 5 if l == 5 else co))
        if g.random() < 0.75:
            c = int(g.integers(0, 5 if l == 0 else ci))
            t = int(g.integers(0, 9))
            wp = [v.copy() for v in weights]
            wm = [v.copy() for v in weights]
            wp[l][o, t, c] += eps
            wm[l][o, t, c] -= eps
            assert gw[l][o, t, c] == pytest.approx((f(wp, biases) - f(wm, biases)) / (2 * eps), rel=1e-5, abs=1e-9)
        else:
            bp = [v.copy() for v in biases]
            bm = [v.copy() for v in biases]
            bp[l][o] += eps
            bm[l][o] -= eps
            assert gb[l][o] == pytest.approx((f(weights, bp) - f(weights, bm)) / (2 * eps), rel=1e-5, abs=1e-9)
    # the one-hop part alone is the one-hop reference
    l1 = cr.net_loss_and_grads(x, t1, weights, biases, dil=dil)[0]
    assert 0 < l1 < loss


def test_adam_first_step_is_lr_times_the_gradient_sign():
    g = np.array([3.0, -0.5, 1e-3, -20.0])
    p1, m, v = cr.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), t=1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1, -0.01 * np.sign(g), rtol=1e-12)

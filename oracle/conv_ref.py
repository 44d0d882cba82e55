"""FP64 reference of the surrogate network's arithmetic: the periodic 3x3
convolution, its two gradients, and the residual six-layer network with its
loss and backward pass.

TEST INFRASTRUCTURE ONLY: the plain, slow restatement that the network's CUDA
kernels (liblbm, lbm_nn_*) are checked against.  Only the test suite loads it.
The paper has no learned component; this file follows the definitions of the
network as the library documents them (include/lbm_nn.h), not its code:

* tap t = 3 (dy + 1) + (dx + 1), dy, dx in {-1, 0, 1};
* conv with dilation d:
         y[n, i, j, o] = b[o] + sum_{t, c} w[o, t, c] x[n, (i + d dy_t) % h, (j + d dx_t) % w, c];
* net:   a_0 = x;  a_{l+1} = max(conv_l(a_l), 0) for l < 5;  out = x + conv_5(a_5),
         layer l with dilation dil[l];
* loss:  mean over pixels and the first `used` channels of (out - target)^2.
"""
from __future__ import annotations

import numpy as np

TAPS = tuple((dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
LAYERS = ((16, 48), (48, 48), (48, 48), (48, 48), (48, 48), (48, 16))


def shifted(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[n, i, j] = x[n, (i + dy) % h, (j + dx) % w]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None, dil: int = 1) -> np.ndarray:
    """x [n, h, w, ci], w [co, 9, ci] -> [n, h, w, co] (float64)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        y += shifted(x, dil * dy, dil * dx) @ w[:, t, :].T
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return y


def conv3x3_dgrad(dy: np.ndarray, w: np.ndarray, dil: int = 1) -> np.ndarray:
    """Gradient with respect to the input: the adjoint of conv3x3 (no bias)."""
    dy = np.asarray(dy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for t, (sy, sx) in enumerate(TAPS):
        dx += shifted(dy @ w[:, t, :], -dil * sy, -dil * sx)
    return dx


def conv3x3_wgrad(x: np.ndarray, dy: np.ndarray, dil: int = 1) -> np.ndarray:
    """dw[o, t, c] = sum over pixels of dy[., o] * x shifted by d times tap t [., c]."""
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    co, ci = dy.shape[3], x.shape[3]
    dw = np.zeros((co, 9, ci))
    d2 = dy.reshape(-1, co)
    for t, (sy, sx) in enumerate(TAPS):
        dw[:, t, :] = d2.T @ shifted(x, dil * sy, dil * sx).reshape(-1, ci)
    return dw


def net_forward(x, weights, biases, dil=(1,) * 6):
    """Activations a_0 .. a_5 and the output of the residual network."""
    acts = [np.asarray(x, dtype=np.float64)]
    for l in range(5):
        acts.append(np.maximum(conv3x3(acts[-1], weights[l], biases[l], dil[l]), 0.0))
    out = acts[0] + conv3x3(acts[5], weights[5], biases[5], dil[5])
    return acts, out


def net_loss_and_grads(x, target, weights, biases, used=5, dil=(1,) * 6):
    """Loss and its gradients with respect to every weight and bias."""
    acts, out = net_forward(x, weights, biases, dil)
    npx = out.shape[0] * out.shape[1] * out.shape[2]
    diff = np.zeros_like(out)
    diff[..., :used] = out[..., :used] - np.asarray(target, dtype=np.float64)[..., :used]
    loss = float((diff ** 2).sum() / (npx * used))
    dz = 2.0 * diff / (npx * used)
    gw, gb = [None] * 6, [None] * 6
    for l in range(5, -1, -1):
        gw[l] = conv3x3_wgrad(acts[l], dz, dil[l])
        gb[l] = dz.sum(axis=(0, 1, 2))
        if l > 0:
            dz = conv3x3_dgrad(dz, weights[l], dil[l]) * (acts[l] > 0.0)
    return loss, gw, gb


def _backward(x, acts, dz, weights, dil):
    """Weight and bias gradients of one network application from the gradient
    dz at its output, and the gradient at its input (residual path plus layer
    0's adjoint)."""
    gw, gb = [None] * 6, [None] * 6
    dout = dz
    for l in range(5, -1, -1):
        gw[l] = conv3x3_wgrad(acts[l], dz, dil[l])
        gb[l] = dz.sum(axis=(0, 1, 2))
        if l > 0:
            dz = conv3x3_dgrad(dz, weights[l], dil[l]) * (acts[l] > 0.0)
        else:
            dz = conv3x3_dgrad(dz, weights[0], dil[0])
    return gw, gb, dout + dz


def net_two_hop_loss_and_grads(x, t1, t2, weights, biases, used=5, dil=(1,) * 6):
    """Loss of two hops unrolled through the network, MSE(net(x), t1) +
    MSE(net(net(x)), t2), and its gradients with respect to every weight and
    bias (the second hop's input gradient flows into the first hop's output)."""
    acts1, out1 = net_forward(x, weights, biases, dil)
    acts2, out2 = net_forward(out1, weights, biases, dil)
    npx = out1.shape[0] * out1.shape[1] * out1.shape[2]

    def mse(out, t):
        d = np.zeros_like(out)
        d[..., :used] = out[..., :used] - np.asarray(t, dtype=np.float64)[..., :used]
        return float((d ** 2).sum() / (npx * used)), 2.0 * d / (npx * used)

    l1, d1 = mse(out1, t1)
    l2, d2 = mse(out2, t2)
    gw2, gb2, dx2 = _backward(out1, acts2, d2, weights, dil)
    gw1, gb1, _ = _backward(x, acts1, d1 + dx2, weights, dil)
    return l1 + l2, [a + b for a, b in zip(gw1, gw2)], [a + b for a, b in zip(gb1, gb2)]


def adam(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma & Ba 2015), float64."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v

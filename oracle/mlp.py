"""FP64 reference of the learned closure network and of its training step.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline may import anything under ``oracle/``.

The closure is not part of the paper.  The paper finds that the SSW scaling
(Sec. 2.4) under-produces sand early in the run and that the coarse model's
drag and cohesion are the terms whose scaling is approximate (Sec. 3); the
closure corrects exactly those two terms per parcel:

* inputs (5): local solid fraction 1 - n_c of the parcel's fluid cell
  (Eq. 6-7), slip speed |u_c - v_i| with u_c = U_s,c / n_c (Eq. 8-11),
  coarse-graining ratio k (Eq. 14), coordination number (active contacts),
  mean overlap delta / d over the active contacts (Eq. 12-13);
* standardisation x_hat = (x - mu) * inv_sigma;
* three hidden layers of 64 SiLU units (silu(z) = z / (1 + exp(-z))), a
  linear output layer of 2 units o;
* corrections c_d = exp(clip(o_1, -c_max, c_max)) multiplying the drag
  force of Eq. 8 and c_g = exp(clip(o_2, -g_max, g_max)) multiplying the
  surface energy of each bond, gamma_ij = gamma sqrt(c_g,i c_g,j) (Eq. 13).

Parameter vector (float): mu[5], inv_sigma[5], then per layer l = 1..4 the
weights W_l[out, in] row by row and the biases b_l[out]; layer sizes
5->64->64->64->2.

Training loss over a batch of B samples with targets y and a 0/1 mask m:
L = 1/(2B) sum_b sum_k m_bk (o_bk - y_bk)^2, minimised by Adam (Kingma and
Ba, 2015: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, step
lr * m_hat / (sqrt(v_hat) + eps) with bias-corrected m_hat, v_hat).

With ``bf16_ops=True`` every operand of a matrix product is rounded to bfloat16
(round to nearest, ties to even) where the tensor-core kernels round it: the
layer inputs (x_hat, h_1, h_2, h_3), the weights, and the back-propagated
pre-activation gradients dZ_l that enter the products dW_l = dZ_l^T a_(l-1)
and dA_(l-1) = dZ_l W_l, and into the bias gradients of the hidden layers
(which the kernels form as the product of dZ_l with a column of ones);
activations, sums and the output layer's bias gradient stay exact here.
"""
from __future__ import annotations

import numpy as np

SIZES = [(5, 64), (64, 64), (64, 64), (64, 2)]
N_IN, N_OUT = 5, 2


def n_params() -> int:
    return 2 * N_IN + sum(o * i + o for i, o in SIZES)


def unpack(theta):
    """Split a parameter vector into (mu, inv_sigma, [(W, b), ...])."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (n_params(),)
    mu, isg = theta[:N_IN], theta[N_IN:2 * N_IN]
    k = 2 * N_IN
    layers = []
    for i, o in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        layers.append((W, b))
    return mu, isg, layers


def pack(mu, isg, layers):
    parts = [np.asarray(mu, np.float64), np.asarray(isg, np.float64)]
    for W, b in layers:
        parts += [np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64)]
    return np.concatenate(parts)


def init_params(seed, mu=None, inv_sigma=None):
    """He-style uniform initialisation (bound sqrt(6 / fan_in) for hidden
    layers, sqrt(1 / fan_in) scaled by 0.1 for the output), zero biases."""
    rng = np.random.default_rng(seed)
    layers = []
    for li, (i, o) in enumerate(SIZES):
        bound = np.sqrt(6.0 / i) if li < len(SIZES) - 1 else 0.1 * np.sqrt(1.0 / i)
        layers.append((rng.uniform(-bound, bound, size=(o, i)), np.zeros(o)))
    return pack(np.zeros(N_IN) if mu is None else mu,
                np.ones(N_IN) if inv_sigma is None else inv_sigma, layers)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    The value is first rounded to float32, the format the kernels hold it in."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _id(a):
    return np.asarray(a, dtype=np.float64)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, bf16_ops=False):
    """Network outputs o [B, 2] and the cache for backward."""
    q = bf16 if bf16_ops else _id
    mu, isg, layers = unpack(theta)
    a = (np.asarray(X, np.float64) - mu) * isg
    acts, zs = [a], []
    for li, (W, b) in enumerate(layers):
        z = q(a) @ q(W).T + b
        zs.append(z)
        a = silu(z) if li < len(layers) - 1 else z
        acts.append(a)
    return a, (acts, zs)


def loss_and_grad(theta, X, Y, M, bf16_ops=False):
    """Loss and its gradient with respect to the weights and biases (the
    standardisation entries of the gradient are zero: they are not trained)."""
    q = bf16 if bf16_ops else _id
    mu, isg, layers = unpack(theta)
    o, (acts, zs) = forward(theta, X, bf16_ops)
    B = len(X)
    r = (o - Y) * M
    L = 0.5 * float((r * (o - Y)).sum()) / B
    dz = r / B
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a_prev = acts[li]
        dzq = q(dz)
        # hidden-layer bias gradients are the product of the rounded dZ with a
        # column of ones; the output layer's is summed from the exact dZ
        db = dz.sum(0) if li == len(layers) - 1 else dzq.sum(0)
        grads[li] = (dzq.T @ q(a_prev), db)
        if li > 0:
            da = dzq @ q(W)
            dz = da * dsilu(zs[li - 1])
    return L, pack(np.zeros(N_IN), np.zeros(N_IN), grads)


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the weights and biases (t counts from 1); the
    standardisation entries are left unchanged."""
    theta = np.array(theta, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    step = lr * mh / (np.sqrt(vh) + eps)
    step[:2 * N_IN] = 0.0
    return theta - step, m, v


def corrections(o, c_max, g_max):
    """(c_d, c_g) from the network outputs."""
    o = np.asarray(o, np.float64)
    return np.exp(np.clip(o[:, 0], -c_max, c_max)), np.exp(np.clip(o[:, 1], -g_max, g_max))

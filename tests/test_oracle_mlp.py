"""Pins of the FP64 closure-network reference (oracle/mlp.py) against values
fixed by mathematics: central finite differences of the loss, a network
built to compute a known composition of SiLU by hand, the bfloat16 rounding
rule of IEEE 754 (round to nearest, ties to even), and Adam's closed-form
first step."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def _silu(z):
    return z / (1.0 + math.exp(-z))


def test_silu_and_derivative():
    assert M.silu(np.array([0.0]))[0] == 0.0
    assert M.dsilu(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    z = np.linspace(-6, 6, 25)
    assert np.allclose(M.silu(z), [_silu(t) for t in z], rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.allclose(M.dsilu(z), fd, rtol=1e-8, atol=1e-9)
    assert M.silu(np.array([40.0]))[0] == pytest.approx(40.0, rel=1e-15)


def test_bf16_rounding_rule():
    e = 2.0 ** -7  # spacing of bfloat16 in [1, 2)
    cases = [
        (1.0, 1.0),
        (1.0 + e / 2, 1.0),                    # tie, even mantissa below
        (1.0 + 1.5 * e, 1.0 + 2 * e),          # tie, even mantissa above
        (1.0 + e / 2 + 2.0 ** -20, 1.0 + e),   # just above the tie
        (1.0 + e / 2 - 2.0 ** -20, 1.0),       # just below the tie
        (-(1.0 + 1.5 * e), -(1.0 + 2 * e)),
        (3.0 * 2.0 ** -130, 3.0 * 2.0 ** -130),  # subnormal float32 held exactly
        (0.0, 0.0),
    ]
    for x, want in cases:
        assert M.bf16(np.array([x]))[0] == want, (x, want)


def test_forward_of_a_hand_built_network():
    """Layer 1 takes x_hat_0 and -x_hat_3 into units 0 and 1, layers 2 and 3
    pass them through as identities, output 0 = 2 h_0 + 0.5, output 1 =
    -h_1.  Then o_0 = 2 silu(silu(silu(s0))) + 0.5 and o_1 = -silu^3(-s3)
    with s = (x - mu) * inv_sigma."""
    mu = np.array([0.1, 0.0, 0.0, -0.3, 0.0])
    isg = np.array([2.0, 1.0, 1.0, 0.5, 1.0])
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in M.SIZES]
    layers[0][0][0, 0] = 1.0
    layers[0][0][1, 3] = -1.0
    for li in (1, 2):
        layers[li][0][0, 0] = 1.0
        layers[li][0][1, 1] = 1.0
    layers[3][0][0, 0] = 2.0
    layers[3][0][1, 1] = -1.0
    layers[3][1][0] = 0.5
    theta = M.pack(mu, isg, layers)
    X = np.random.default_rng(0).normal(size=(7, 5))
    o, _ = M.forward(theta, X)
    for b in range(7):
        s0 = (X[b, 0] - mu[0]) * isg[0]
        s3 = (X[b, 3] - mu[3]) * isg[3]
        assert o[b, 0] == pytest.approx(2 * _silu(_silu(_silu(s0))) + 0.5, rel=1e-14)
        assert o[b, 1] == pytest.approx(-_silu(_silu(_silu(-s3))), rel=1e-13, abs=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = M.init_params(3, mu=rng.normal(size=5), inv_sigma=rng.uniform(0.5, 2, 5))
    theta[2 * M.N_IN:] += 0.05 * rng.normal(size=M.n_params() - 2 * M.N_IN)  # nonzero biases
    X = rng.normal(size=(16, 5))
    Y = rng.normal(size=(16, 2))
    Mk = (rng.uniform(size=(16, 2)) < 0.8).astype(float)
    L, g = M.loss_and_grad(theta, X, Y, Mk)
    assert np.all(g[:2 * M.N_IN] == 0)
    idx = np.concatenate([rng.choice(np.arange(2 * M.N_IN, M.n_params()), 400, replace=False),
                          np.arange(M.n_params() - 130, M.n_params())])  # all of layer 4
    h = 1e-5  # truncation ~h^2, rounding ~1e-16 L / h: both below 1e-10 here
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_and_grad(tp, X, Y, Mk)[0] - M.loss_and_grad(tm, X, Y, Mk)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-10), k


def test_zero_output_weights_give_bias_and_mean_residual():
    rng = np.random.default_rng(2)
    theta = M.init_params(4)
    mu, isg, layers = M.unpack(theta)
    layers[3] = (np.zeros((2, 64)), np.array([0.25, -1.0]))
    theta = M.pack(mu, isg, layers)
    X = rng.normal(size=(9, 5))
    Y = rng.normal(size=(9, 2))
    Mk = np.ones((9, 2))
    o, _ = M.forward(theta, X)
    assert np.all(o == np.array([0.25, -1.0]))
    L, g = M.loss_and_grad(theta, X, Y, Mk)
    assert L == pytest.approx(0.5 * ((o - Y) ** 2).sum() / 9, rel=1e-14)
    gb4 = g[-2:]
    assert gb4 == pytest.approx((o - Y).mean(0), rel=1e-14)
    # nothing flows below a zero output layer
    assert np.all(g[2 * M.N_IN:M.n_params() - 130] == 0)


def test_perfect_fit_has_zero_loss_and_gradient():
    theta = M.init_params(5)
    X = np.random.default_rng(3).normal(size=(11, 5))
    Y, _ = M.forward(theta, X)
    L, g = M.loss_and_grad(theta, X, Y, np.ones_like(Y))
    assert L == 0.0 and np.all(g == 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    theta = rng.normal(size=M.n_params())
    g = rng.normal(size=M.n_params())
    g[:2 * M.N_IN] = 0
    lr, eps = 1e-3, 1e-8
    t1, m, v = M.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr, eps=eps)
    want = theta - lr * g / (np.abs(g) + eps)
    want[:2 * M.N_IN] = theta[:2 * M.N_IN]
    assert np.allclose(t1, want, rtol=1e-13, atol=1e-16)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_gradient_is_near_the_exact_one():
    rng = np.random.default_rng(7)
    theta = M.init_params(8)
    X = rng.normal(size=(64, 5))
    Y = rng.normal(size=(64, 2))
    Mk = np.ones((64, 2))
    _, g = M.loss_and_grad(theta, X, Y, Mk)
    _, gq = M.loss_and_grad(theta, X, Y, Mk, bf16_ops=True)
    rel = np.linalg.norm(gq - g) / np.linalg.norm(g)
    assert 1e-5 < rel < 2.0 ** -5  # rounded, but only at the bfloat16 level


def test_corrections_clip():
    o = np.array([[0.0, 0.0], [10.0, -10.0], [-1.0, 0.5]])
    cd, cg = M.corrections(o, 3.0, math.log(4))
    assert cd == pytest.approx([1.0, math.exp(3.0), math.exp(-1.0)])
    assert cg == pytest.approx([1.0, 0.25, math.exp(0.5)])

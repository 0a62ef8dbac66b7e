"""The closure network's tensor-core kernels (through the C ABI) against the
FP64 reference in oracle/mlp.py.

The reference runs in its bfloat16 mode: it rounds to bfloat16 exactly the
operands the kernels round (standardised inputs, activations, weights,
back-propagated gradients), so the two differ only by the kernels' FP32
accumulation and by the rare activation whose FP32 value sits so close to a
bfloat16 rounding boundary that the two sides round it apart (one bfloat16
step, 2^-8 relative, in one element).  Tolerances:
* outputs: median error <= 1e-5 and every error <= 2^-6 of the output's
  term-magnitude sum S = sum_j |W4_kj h3_j| + |b4_k|;
* gradients: normwise relative error per layer <= 1e-3;
* Adam: the updated parameters follow the reference's Adam on the
  reference's gradient within 1e-3 of the step size wherever the gradient is
  not tiny (where it is, Adam's step sign is decided by rounding noise).
Sample counts cover a single partial tile, a ragged tail, and more tiles
than SMs (tiles accumulated in one CTA).
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2211_06142_gb300 import cgdem

pytestmark = pytest.mark.gpu


def make_theta(seed):
    rng = np.random.default_rng(seed)
    theta = M.init_params(seed, mu=rng.normal(0, 0.5, 5), inv_sigma=rng.uniform(0.5, 2.0, 5))
    theta[2 * M.N_IN:] += 0.02 * rng.normal(size=M.n_params() - 2 * M.N_IN)
    # the kernels hold FP32 parameters: the reference uses the same values
    return theta.astype(np.float32).astype(np.float64)


def make_data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 5)).astype(np.float32).astype(np.float64)
    Y = rng.normal(size=(n, 2)).astype(np.float32).astype(np.float64)
    Mk = (rng.uniform(size=(n, 2)) < 0.85).astype(np.float64)
    return X, Y, Mk


def out_scale(theta, X):
    _, (acts, _) = M.forward(theta, X, bf16_ops=True)
    _, _, layers = M.unpack(theta)
    W4, b4 = layers[3]
    return np.abs(M.bf16(acts[3])) @ np.abs(M.bf16(W4)).T + np.abs(b4)


@pytest.mark.parametrize("n", [77, 1000, 2 * 128 * 160 + 5])
def test_forward_matches_reference(n):
    theta = make_theta(1)
    X, _, _ = make_data(n, 2)
    net = cgdem.Closure(theta)
    o = net.forward(X).cpu().numpy().astype(np.float64)
    ref, _ = M.forward(theta, X, bf16_ops=True)
    S = out_scale(theta, X)
    err = np.abs(o - ref) / S
    assert np.median(err) <= 1e-5, np.median(err)
    assert err.max() <= 2.0 ** -6, err.max()
    exact, _ = M.forward(theta, X)
    assert (np.abs(o - exact) / S).max() <= 2.0 ** -3  # bfloat16-level distance from exact math


def layer_slices():
    k = 2 * M.N_IN
    out = []
    for i, o in M.SIZES:
        out.append(slice(k, k + o * i + o))
        k += o * i + o
    return out


@pytest.mark.parametrize("n", [77, 1000, 2 * 128 * 160 + 5])
def test_gradient_matches_reference(n):
    theta = make_theta(3)
    X, Y, Mk = make_data(n, 4)
    net = cgdem.Closure(theta)
    L, g = net.gradient(X, Y, Mk)
    g = g.cpu().numpy().astype(np.float64)
    Lr, gr = M.loss_and_grad(theta, X, Y, Mk, bf16_ops=True)
    assert L == pytest.approx(Lr, rel=1e-4)
    assert np.all(g[:2 * M.N_IN] == 0)
    for li, sl in enumerate(layer_slices()):
        rel = np.linalg.norm(g[sl] - gr[sl]) / np.linalg.norm(gr[sl])
        assert rel <= 1e-3, (li, rel)


def test_adam_steps_match_reference():
    theta = make_theta(5)
    X, Y, Mk = make_data(3000, 6)
    net = cgdem.Closure(theta)
    lr = 1e-3
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 4):
        hist = net.train(X, Y, Mk, 1, lr)
        L, g = M.loss_and_grad(th, X, Y, Mk, bf16_ops=True)
        assert hist[0] == pytest.approx(L, rel=1e-3)
        th, m, v = M.adam_step(th, g, m, v, t, lr)
        got = net.params().astype(np.float64)
        assert np.array_equal(got[:2 * M.N_IN], theta[:2 * M.N_IN].astype(np.float32))
        big = np.abs(g) > 1e-2 * np.abs(g).max()
        assert big.sum() > 200
        assert np.abs(got - th)[big].max() <= 1e-3 * lr * t + 1e-6 * np.abs(th[big]).max()
        # where the gradient is tiny Adam still moves by at most lr per step
        assert np.abs(got - theta).max() <= 3 * t * lr + 1e-6


def test_training_reduces_loss_like_the_reference():
    """Fit a fixed teacher network: 200 full-batch Adam steps on the GPU end
    at a loss within a factor 1.5 of the same 200 steps taken by the FP64
    reference (no bfloat16), and more than 10x below the initial loss."""
    rng = np.random.default_rng(9)
    teacher = M.init_params(11)
    teacher[-130:] *= 20.0  # outputs of order one
    X = rng.normal(size=(4096, 5)).astype(np.float32).astype(np.float64)
    Y, _ = M.forward(teacher, X)
    Y = Y.astype(np.float32).astype(np.float64)
    Mk = np.ones_like(Y)
    theta = make_theta(12)
    net = cgdem.Closure(theta)
    hist = net.train(X, Y, Mk, 200, 3e-3)
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    L0 = None
    for t in range(1, 201):
        L, g = M.loss_and_grad(th, X, Y, Mk)
        L0 = L if L0 is None else L0
        th, m, v = M.adam_step(th, g, m, v, t, 3e-3)
    Lref, _ = M.loss_and_grad(th, X, Y, Mk)
    Lgpu, _ = M.loss_and_grad(net.params().astype(np.float64), X, Y, Mk)
    assert hist[0] == pytest.approx(L0, rel=2e-2)
    assert Lref < 0.1 * L0
    assert Lgpu < 0.1 * L0
    assert Lgpu <= 1.5 * Lref, (Lgpu, Lref, L0)

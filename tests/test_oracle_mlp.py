"""Pins of the FP64 network oracle (oracle/mlp.py) used to check the GPU training kernels.

The hand-written backward pass is checked against central finite differences of the loss
(a different computation: only the forward pass enters), a one-neuron network is checked
against values worked out by hand, and the Adam step against its first-step closed form.
"""
import numpy as np

from oracle import mlp


def _loss(params, x, t):
    y, _ = mlp.forward(params, x)
    return np.sum((y - t) ** 2) / y.size


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    sizes = [5, 7, 6, 4]
    params = mlp.init(sizes, seed=2)
    params = [p + 0.1 * rng.normal(size=p.shape) for p in params]  # nonzero biases too
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 4))
    loss, grads = mlp.loss_and_grads(params, x, t)
    assert abs(loss - _loss(params, x, t)) < 1e-15
    h = 1e-6
    for p, g in zip(params, grads):
        assert g.shape == p.shape
        fd = np.zeros_like(p)
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + h
            lp = _loss(params, x, t)
            p[idx] = old - h
            lm = _loss(params, x, t)
            p[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        assert np.abs(fd - g).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_one_neuron_by_hand():
    # y = w2 tanh(w1 x + b1) + b2 with x = 1, t = 0
    w1, b1, w2, b2 = 0.5, 0.25, 2.0, -1.0
    params = [np.array([[w1]]), np.array([b1]), np.array([[w2]]), np.array([b2])]
    x, t = np.array([[1.0]]), np.array([[0.0]])
    a = np.tanh(0.75)
    y = 2.0 * a - 1.0
    loss, (gw1, gb1, gw2, gb2) = mlp.loss_and_grads(params, x, t)
    assert abs(loss - y * y) < 1e-15
    dy = 2.0 * y
    assert abs(gb2[0] - dy) < 1e-15 and abs(gw2[0, 0] - dy * a) < 1e-15
    dz = dy * w2 * (1.0 - a * a)
    assert abs(gb1[0] - dz) < 1e-15 and abs(gw1[0, 0] - dz * 1.0) < 1e-15


def test_linear_network_gradient_closed_form():
    # one linear layer: grad_W = 2/n (X W^T + b - T)^T X, grad_b = 2/n sum of the rows
    rng = np.random.default_rng(5)
    W, b = rng.normal(size=(3, 4)), rng.normal(size=3)
    x, t = rng.normal(size=(6, 4)), rng.normal(size=(6, 3))
    _, (gW, gb) = mlp.loss_and_grads([W, b], x, t)
    R = x @ W.T + b - t
    assert np.allclose(gW, 2.0 / R.size * R.T @ x, rtol=0, atol=1e-14)
    assert np.allclose(gb, 2.0 / R.size * R.sum(axis=0), rtol=0, atol=1e-14)


def test_adam_first_step_is_signed_lr():
    # after bias correction the first step is -lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    assert np.allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_standardize_and_fold_closed_forms():
    """Standardised columns have mean 0 and population standard deviation 1 (a constant column
    becomes 0), and the folded layer returns scale * (W x + b) + mean for any x."""
    rng = np.random.default_rng(5)
    T = rng.normal(3.0, 2.0, size=(40, 6))
    T[:, 2] = 7.5
    mean, scale, Tn = mlp.standardize(T)
    assert np.allclose(Tn.mean(axis=0), 0.0, atol=1e-14)
    sd = Tn.std(axis=0)
    assert np.allclose(np.delete(sd, 2), 1.0, atol=1e-14) and np.all(Tn[:, 2] == 0.0)
    assert scale[2] == 1.0 and mean[2] == 7.5
    W, b = rng.normal(size=(6, 4)), rng.normal(size=6)
    Wf, bf = mlp.fold_affine(W, b, mean, scale)
    x = rng.normal(size=4)
    assert np.allclose(Wf @ x + bf, scale * (W @ x + b) + mean, rtol=1e-14, atol=1e-14)

"""FP64 reference of the small network used for the learned PCG initial guess
(oracle; test infrastructure).

x -> tanh(x W1^T + b1) -> tanh(. W2^T + b2) -> . W3^T + b3, loss = mean((y - t)^2).
Forward and backward are written out directly (chain rule by hand) and Adam follows its
published update; pinned in the tests by central finite differences, a one-neuron case worked
out by hand and Adam's first-step closed form.
"""

import numpy as np


def init(sizes, seed=7):
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(sizes) - 1):
        fan_in = sizes[i]
        W = rng.normal(0.0, 1.0 / np.sqrt(fan_in), size=(sizes[i + 1], sizes[i]))
        b = np.zeros(sizes[i + 1])
        params += [W, b]
    return params


def forward(params, x):
    """Returns (output, activations) with activations[i] the input of layer i."""
    acts = [x]
    h = x
    nl = len(params) // 2
    for i in range(nl):
        W, b = params[2 * i], params[2 * i + 1]
        z = h @ W.T + b
        h = np.tanh(z) if i < nl - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grads(params, x, t):
    y, acts = forward(params, x)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    grads = [None] * len(params)
    nl = len(params) // 2
    dz = dy
    for i in reversed(range(nl)):
        W = params[2 * i]
        h_in = acts[i]
        grads[2 * i] = dz.T @ h_in
        grads[2 * i + 1] = dz.sum(axis=0)
        if i > 0:
            dh = dz @ W
            dz = dh * (1.0 - acts[i] ** 2)  # tanh'(z) = 1 - tanh(z)^2
    return loss, grads


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) with bias-corrected moments."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def standardize(T):
    """Column statistics of the training targets T [M, N]: mean, scale (population standard
    deviation, 1 for a column with zero spread) and the standardised targets (T - mean) / scale."""
    mean = T.mean(axis=0)
    sd = np.sqrt(((T - mean) ** 2).mean(axis=0))
    scale = np.where(sd > 0, sd, 1.0)
    return mean, scale, (T - mean) / scale


def fold_affine(W, b, mean, scale):
    """The last layer y = W x + b trained on standardised targets, rewritten to return the
    targets: W' = diag(scale) W, b' = scale * b + mean."""
    return W * scale[:, None], b * scale + mean

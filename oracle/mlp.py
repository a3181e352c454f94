"""FP64 reference of the surrogate network (test infrastructure only).

A multilayer perceptron maps the stochastic process inputs (melt
temperature, wall temperature, solute concentration; Section 2.7 treats
such inputs as random variables) to the microstructure outputs of
Section 2.6 (Eq. 22-23).  Layers: x -> GELU(W1 x + b1) -> ... -> W_L h + b_L
(linear output), mean-squared-error loss.  GELU(z) = z Phi(z) with Phi the
standard normal distribution function.

Parameters are a list of (W [n_out, n_in], b [n_out]) in FP64.  Only the
tests, the smoke entry point and the benchmark's CPU leg use this file.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def gelu(z):
    """GELU(x) = x Phi(x), the surrogate's activation (the surrogate is not in the paper; it stands in for the collocation fits of Section 2.7 inside the Monte Carlo loop)."""
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """Derivative of GELU: Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(sizes, seed):
    """He-style uniform initialisation (the GPU uses its own counter-based
    generator; tests pass parameters explicitly)."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / a)
        params.append((rng.uniform(-lim, lim, (b, a)), np.zeros(b)))
    return params


def forward(params, X):
    """Returns (output, cache) with the pre-activations and activations."""
    hs, zs = [X], []
    h = X
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = z if i == len(params) - 1 else gelu(z)
        hs.append(h)
    return h, (hs, zs)


def loss(params, X, Y):
    """Mean squared error over batch and outputs."""
    out, _ = forward(params, X)
    return np.mean((out - Y) ** 2)


def backward(params, X, Y):
    """Gradients of the mean-squared error (mean over batch and outputs)."""
    out, (hs, zs) = forward(params, X)
    n = out.size
    d = 2.0 * (out - Y) / n
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        grads[i] = (d.T @ hs[i], d.sum(axis=0))
        if i > 0:
            d = (d @ W) * gelu_grad(zs[i - 1])
    return grads


def flatten(params):
    """Parameter packing (no arithmetic)."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, sizes):
    """Parameter unpacking (no arithmetic)."""
    params, k = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = vec[k:k + a * b].reshape(b, a)
        k += a * b
        params.append((W, vec[k:k + b].copy()))
        k += b
    return params


def adam_init(n):
    """Adam state for n parameters: first and second moments at zero, step 0."""
    return dict(m=np.zeros(n), v=np.zeros(n), t=0)


def adam_step(state, theta, g, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) of the flat
    parameters theta with gradient g: exponential moving averages of g and
    g^2, each divided by (1 - beta^t) to remove the bias of the zero start,
    then theta - lr m_hat / (sqrt(v_hat) + eps).  Returns the new parameters
    and updates the state in place."""
    state["t"] += 1
    t = state["t"]
    state["m"] = beta1 * state["m"] + (1.0 - beta1) * g
    state["v"] = beta2 * state["v"] + (1.0 - beta2) * g * g
    m_hat = state["m"] / (1.0 - beta1 ** t)
    v_hat = state["v"] / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps)

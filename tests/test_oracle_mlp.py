"""Pins of the FP64 surrogate reference: central finite differences of the
loss (h = 1e-6) match the analytic gradients; GELU against its definition
z Phi(z) at known points."""
import numpy as np

from oracle.mlp import backward, flatten, gelu, gelu_grad, init_params, loss, unflatten


def test_gelu_known_values():
    # Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (standard normal table)
    assert gelu(0.0) == 0.0
    assert abs(gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(gelu(-1.0) + 1.0 - 0.8413447460685429) < 1e-15
    z = np.linspace(-4, 4, 81)
    fd = (gelu(z + 1e-6) - gelu(z - 1e-6)) / 2e-6
    assert np.abs(fd - gelu_grad(z)).max() < 1e-8


def test_gradients_match_finite_differences():
    sizes = [3, 16, 16, 4]
    p = init_params(sizes, 3)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(20, 3))
    Y = rng.normal(size=(20, 4))
    g = flatten([(gW, gb) for gW, gb in backward(p, X, Y)])
    v = flatten(p)
    idx = rng.choice(len(v), 40, replace=False)
    for i in idx:
        e = np.zeros_like(v)
        e[i] = 1e-6
        fd = (loss(unflatten(v + e, sizes), X, Y) - loss(unflatten(v - e, sizes), X, Y)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])

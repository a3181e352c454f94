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


def test_adam_first_step_closed_form():
    """With the bias correction the first Adam step is -lr g/(|g| + eps)
    whatever beta1 and beta2 are (m_hat = g, v_hat = g^2).  Dropping either
    correction scales the step by 0.1 or by 1/sqrt(0.001), and a wrong sign
    reverses it; each of these fails here (planted and checked)."""
    from oracle.mlp import adam_init, adam_step
    rng = np.random.default_rng(5)
    g = rng.normal(size=50) * np.logspace(-6, 2, 50)
    th0 = rng.normal(size=50)
    for b1, b2 in ((0.9, 0.999), (0.5, 0.9)):
        st = adam_init(50)
        th1 = adam_step(st, th0, g, 1e-3, b1, b2, 1e-8)
        np.testing.assert_allclose(th1 - th0, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_adam_second_step_closed_forms():
    """Second step: a repeated gradient gives the same step again
    (m_hat = g, v_hat = g^2 once more); a reversed gradient gives
    m_hat = -(1 - b1) g/(1 + b1) and v_hat = g^2, i.e. a step of
    +lr (1 - b1)/(1 + b1) sign(g) (0.1/1.9 for b1 = 0.9)."""
    from oracle.mlp import adam_init, adam_step
    rng = np.random.default_rng(6)
    g = rng.normal(size=40) + np.sign(rng.normal(size=40))
    th0 = rng.normal(size=40)
    st = adam_init(40)
    th1 = adam_step(st, th0, g, 1e-2)
    th2 = adam_step(st, th1, g, 1e-2)
    np.testing.assert_allclose(th2 - th1, th1 - th0, rtol=1e-9, atol=1e-15)
    st = adam_init(40)
    th1 = adam_step(st, th0, g, 1e-2)
    th2 = adam_step(st, th1, -g, 1e-2, eps=0.0)
    np.testing.assert_allclose(th2 - th1, 1e-2 * (0.1 / 1.9) * np.sign(g), rtol=1e-12)

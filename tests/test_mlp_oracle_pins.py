"""Pins of the oracle's FP64 network backprop: central differences of the loss,
and closed forms for nets whose hidden layers are switched off."""
import numpy as np

from oracle import mlp as M


def _params(k, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.3, M.n_params(k))


def test_backprop_matches_central_differences():
    for k in (1, 5):
        p = _params(k, 1 + k)
        rng = np.random.default_rng(7)
        x = rng.uniform(-1, 1, 37)
        y = rng.uniform(-1, 1, (k, 37))
        _, g = M.loss_and_grad(p, k, x, y)
        idx = rng.choice(p.size, 60, replace=False)
        for i in idx:
            h = 1e-6
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (M.loss_and_grad(pp, k, x, y)[0] - M.loss_and_grad(pm, k, x, y)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (k, i, fd, g[i])


def test_output_bias_only_net_has_the_closed_form_gradient():
    k, n = 3, 11
    p = np.zeros(M.n_params(k))
    p[-k:] = [0.5, -0.25, 1.0]                     # y = b3 everywhere (W3 = 0)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, n)
    y = rng.uniform(-1, 1, (k, n))
    loss, g = M.loss_and_grad(p, k, x, y)
    b3 = p[-k:]
    assert np.allclose(loss, np.mean((b3[:, None] - y) ** 2), rtol=1e-14)
    assert np.allclose(g[-k:], 2.0 * (b3 - y.mean(axis=1)) / k, rtol=1e-13)
    assert np.all(g[:-k] == 0.0)                    # nothing upstream of a zero W3 moves the loss


def test_forward_of_a_linear_regime_net():
    """Tiny weights: tanh is linear to first order, so y ~ W3 (W2 (W1 x + b1) + b2) + b3."""
    k = 2
    p = _params(k, 5) * 1e-4
    x = np.linspace(-1, 1, 9)
    W1, b1, W2, b2, W3, b3 = M.unpack(p, k)
    lin = W3 @ (W2 @ (np.outer(W1, x) + b1[:, None]) + b2[:, None]) + b3[:, None]
    assert np.allclose(M.forward(p, k, x), lin, rtol=0, atol=1e-14)

"""Pins of the oracle's SIREN (the neural field): reverse-mode gradients and forward-mode
Jacobians against central finite differences, the MSE value against its definition, and
Adam's first step against its closed form (update = lr g / (|g| + eps))."""
import numpy as np

from oracle import siren
from paper_2403_06706_gb300 import synth

RNG = np.random.default_rng(8)
W0 = 30.0


def _small_params():
    # the full width is 256; the pins use the real shapes with a few samples
    return synth.siren_init(seed=1).astype(np.float64)


def test_param_layout_and_count():
    p = _small_params()
    assert p.size == siren.n_params() == 200456
    d = siren.unpack(p)
    assert d["W2"].shape == (256, 256) and d["W5"].shape == (8, 256) and d["b5"].shape == (8,)
    np.testing.assert_array_equal(siren.pack(d), p)


def test_jacobian_matches_finite_differences():
    p = _small_params()
    x = RNG.uniform(-0.9, 0.9, (5, 3))
    y, J = siren.forward(p, x, W0, jac=True)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (siren.forward(p, x + e, W0) - siren.forward(p, x - e, W0)) / (2 * h)
        np.testing.assert_allclose(J[:, :, j], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    np.testing.assert_allclose(siren.forward(p, x, W0), y, rtol=0, atol=0)


def test_gradient_matches_finite_differences():
    p = _small_params()
    x = RNG.uniform(-0.9, 0.9, (7, 3))
    t = RNG.normal(size=(7, 8))
    L, g = siren.loss_and_grad(p, x, t, W0)
    y = siren.forward(p, x, W0)
    assert abs(L - np.mean((y - t) ** 2)) < 1e-14 * max(1.0, L)
    idx = np.concatenate([RNG.choice(768, 6, replace=False),            # W1
                          768 + RNG.choice(256, 3, replace=False),      # b1
                          1024 + RNG.choice(65536, 6, replace=False),   # W2
                          p.size - 8 - 2048 + RNG.choice(2048, 4, replace=False),  # W5
                          p.size - 8 + np.arange(3)])                   # b5
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (siren.loss_and_grad(pp, x, t, W0)[0] - siren.loss_and_grad(pm, x, t, W0)[0]) / (2 * h)
        assert abs(g[i] - fd) < 1e-6 * max(abs(fd), 1e-4), (i, g[i], fd)


def test_adam_first_step_closed_form():
    theta = RNG.normal(size=10)
    g = RNG.normal(size=10)
    lr, eps = 1e-3, 1e-8
    out, m, v = siren.adam_step(theta, g, np.zeros(10), np.zeros(10), 1, lr, eps=eps)
    np.testing.assert_allclose(out, theta - lr * g / (np.abs(g) + eps), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_init_is_sitzmann():
    d = siren.unpack(synth.siren_init(seed=2).astype(np.float64))
    assert np.abs(d["W1"]).max() <= 1 / 3
    assert np.abs(d["W3"]).max() <= np.sqrt(6 / 256)
    assert np.abs(d["W5"]).max() <= np.sqrt(6 / 256) / 30
    # hidden pre-activations stay O(1): sin of them is roughly arcsine-distributed
    x = RNG.uniform(-1, 1, (2000, 3))
    p = synth.siren_init(seed=2).astype(np.float64)
    dd = siren.unpack(p)
    h = np.sin(W0 * (x @ dd["W1"].T + dd["b1"]))
    z = h @ dd["W2"].T + dd["b2"]
    assert 0.5 < z.std() < 2.0

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


def test_round_bf16_matches_torch_and_ties_to_even():
    torch = __import__("pytest").importorskip("torch")
    v = RNG.normal(size=20000).astype(np.float32) * np.float32(10.0) ** RNG.integers(-6, 6, 20000)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(siren.round_bf16(v.astype(np.float64)), ref)
    # halfway cases go to the even neighbour: 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    np.testing.assert_array_equal(siren.round_bf16([1 + 2.0**-8, 1 + 3 * 2.0**-8, -(1 + 2.0**-8)]),
                                  [1.0, 1 + 2.0**-6, -1.0])


def test_bf16_reading_is_close_to_the_exact_network():
    p = _small_params()
    x = RNG.uniform(-0.9, 0.9, (50, 3))
    y, J = siren.forward(p, x, W0, jac=True)
    yb, Jb = siren.forward(p, x, W0, jac=True, bf16=True)
    assert np.sqrt(np.mean((yb - y) ** 2)) < 0.05 * np.sqrt(np.mean(y**2))
    assert np.sqrt(np.mean((Jb - J) ** 2)) < 0.05 * np.sqrt(np.mean(J**2))
    assert np.abs(yb - y).max() > 0  # the reading does round


def _linear_grid(n_ph=8, n_th=6, n_r=5):
    # node values linear in the index coordinates (i, j, k) of each node
    k, j, i = np.meshgrid(np.arange(n_ph), np.arange(n_th), np.arange(n_r), indexing="ij")
    coef = RNG.normal(size=(8, 4))
    return np.stack([coef[c, 0] + coef[c, 1] * i + coef[c, 2] * j + coef[c, 3] * k for c in range(8)], -1), coef


def test_grid_targets_reproduce_nodes_and_index_linear_fields():
    nodes, coef = _linear_grid()
    n_ph, n_th, n_r = nodes.shape[:3]
    r_min, r_max = 0.1 * siren.AU, 2.5 * siren.AU
    dr = (r_max - r_min) / (n_r - 1)
    # random points strictly inside (no phi wrap: k + fp < n_ph - 1)
    xi = RNG.uniform(0, n_r - 1, 200)
    xt = RNG.uniform(0.01, n_th - 1.01, 200)
    xp = RNG.uniform(0, n_ph - 1.01, 200)
    r, th, ph = r_min + xi * dr, xt * np.pi / (n_th - 1), xp * 2 * np.pi / n_ph
    R = np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], 1)
    t = siren.grid_targets(nodes, r_min, r_max, R / r_max, r_max, 1.0, 1.0)
    lin = coef[:, 0] + np.outer(xi, coef[:, 1]) + np.outer(xt, coef[:, 2]) + np.outer(xp, coef[:, 3])
    a = r / siren.AU
    expect = lin * np.stack([a**2] * 3 + [a] * 3 + [a**2, 1 / siren.AU * np.ones_like(a)], 1)
    np.testing.assert_allclose(t, expect, rtol=1e-9, atol=1e-12)


def test_grid_targets_agree_with_the_c_oracle_gather():
    import oracle
    w = synth.WindSpec(16, 12, 16, eps=0.1, n_modes=4)
    nodes = synth.wind_grid(w, dtype=np.float64)
    f = oracle.grid_field(nodes, w.r_min_au * siren.AU, w.r_max_au * siren.AU)
    r = RNG.uniform(0.2, 2.3, 40) * siren.AU
    th = np.arccos(RNG.uniform(-0.95, 0.95, 40))
    ph = RNG.uniform(0, 2 * np.pi, 40)
    R = np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], 1)
    t = siren.grid_targets(nodes, w.r_min_au * siren.AU, w.r_max_au * siren.AU, R / (2.5 * siren.AU),
                           2.5 * siren.AU, w.B1, w.B1 * w.u_sw)
    for q in range(40):
        s, _ = oracle.field_eval(f, R[q])
        a = r[q] / siren.AU
        np.testing.assert_allclose(t[q, 0:3], s["B"] * a * a / w.B1, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(t[q, 3:6], s["E"] * a / (w.B1 * w.u_sw), rtol=1e-9, atol=1e-12)


def test_physical_field_is_the_derivative_of_the_unscaled_network():
    p = _small_params()
    rs, Bs, Es = 2.5 * siren.AU, 3.5e-9, 1.4e-3
    x = RNG.uniform(-0.8, 0.8, (4, 3))
    y, J = siren.forward(p, x, W0, jac=True)
    B, E, dB, dE = siren.physical_field(x, y, J, rs, Bs, Es)

    def BE(R):
        xx = R / rs
        yy, JJ = siren.forward(p, xx, W0, jac=True)
        b, e, _, _ = siren.physical_field(xx, yy, JJ, rs, Bs, Es)
        return b, e

    h = 1e-7 * rs
    for d in range(3):
        e_ = np.zeros(3)
        e_[d] = h
        bp, ep = BE(x * rs + e_)
        bm, em = BE(x * rs - e_)
        np.testing.assert_allclose(dB[:, d, :], (bp - bm) / (2 * h), rtol=1e-5, atol=1e-6 * np.abs(dB).max())
        np.testing.assert_allclose(dE[:, d, :], (ep - em) / (2 * h), rtol=1e-5, atol=1e-6 * np.abs(dE).max())


def test_c_oracle_neural_field_matches_numpy_reading():
    """The C oracle's neural field (used by its push) against the numpy reading above, in
    both arithmetics, and its Jacobians against finite differences of its own values."""
    import oracle
    p = _small_params()
    rs, Bs, Es = 2.5 * siren.AU, 3.5e-9, 1.4e-3
    for bf16 in (False, True):
        f = oracle.siren_field(p, W0, rs, Bs, Es, bf16=bf16)
        x = RNG.uniform(-0.8, 0.8, (6, 3))
        y, J = siren.forward(p, x, W0, jac=True, bf16=bf16)
        B, E, dB, dE = siren.physical_field(x, y, J, rs, Bs, Es)
        for q in range(6):
            s, fl = oracle.field_eval(f, x[q] * rs)
            assert fl == 0
            np.testing.assert_allclose(s["B"], B[q], rtol=1e-10, atol=1e-12 * np.abs(B).max())
            np.testing.assert_allclose(s["E"], E[q], rtol=1e-10, atol=1e-12 * np.abs(E).max())
            # oracle JB[c][d] = dB_c / dR_d; physical_field dB[d][c]
            np.testing.assert_allclose(s["JB"], dB[q].T, rtol=1e-9, atol=1e-12 * np.abs(dB).max())
            np.testing.assert_allclose(s["JE"], dE[q].T, rtol=1e-9, atol=1e-12 * np.abs(dE).max())
    f = oracle.siren_field(p, W0, rs, Bs, Es)
    R = np.array([0.4, -0.3, 0.2]) * rs
    s0, _ = oracle.field_eval(f, R)
    h = 1e-6 * rs
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        sp, _ = oracle.field_eval(f, R + e)
        sm, _ = oracle.field_eval(f, R - e)
        np.testing.assert_allclose(s0["JB"][:, d], (sp["B"] - sm["B"]) / (2 * h), rtol=1e-5,
                                   atol=1e-6 * np.abs(s0["JB"]).max())

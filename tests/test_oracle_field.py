"""Pins of the oracle's field evaluation (trilinear interpolation, Sect. 2.2) and of its
analytic fields, plus checks of the synthetic wind generator.

Independent references: exactness of trilinear interpolation at nodes and for data
that are linear in index space, Cartesian finite differences of closed-form
coordinate maps, convergence orders of interpolation (O(h^2) values, O(h)
gradients), and vector identities (div B = 0, curl E = 0, E.B = 0).
"""
import numpy as np
import pytest

import oracle
from oracle import AU
from paper_2403_06706_gb300 import synth

RNG = np.random.default_rng(1234)


def node_xyz(r, th, ph):
    return np.array([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)])


def grid_axes(nr, nt, npf, rmin, rmax):
    r = rmin + (rmax - rmin) * np.arange(nr) / (nr - 1)
    th = np.pi * np.arange(nt) / (nt - 1)
    ph = 2 * np.pi * np.arange(npf) / npf
    return r, th, ph


def test_interpolant_equals_node_values():
    nr, nt, npf = 9, 7, 10
    rmin, rmax = 0.2 * AU, 1.8 * AU
    nodes = RNG.normal(size=(npf, nt, nr, 8))
    f = oracle.grid_field(nodes, rmin, rmax)
    r, th, ph = grid_axes(nr, nt, npf, rmin, rmax)
    for _ in range(60):
        i, j, k = RNG.integers(0, nr), RNG.integers(1, nt - 1), RNG.integers(0, npf)
        out, fl = oracle.field_eval(f, node_xyz(r[i], th[j], ph[k]))
        assert fl == 0
        np.testing.assert_allclose(out["B"], nodes[k, j, i, 0:3], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(out["E"], nodes[k, j, i, 3:6], rtol=1e-9, atol=1e-12)


def _coords(X, rmin, dr, dth, dph):
    x, y, z = X
    r = np.sqrt(x * x + y * y + z * z)
    th = np.arctan2(np.hypot(x, y), z)
    ph = np.arctan2(y, x) % (2 * np.pi)
    return (r - rmin) / dr, th / dth, ph / dph


def test_linear_in_index_data_exact_values_and_cartesian_gradient():
    """Node data a + b i + c j + d k are reproduced exactly by a trilinear interpolant;
    the chain rule to Cartesian derivatives is checked against central differences of the
    closed-form coordinate maps."""
    nr, nt, npf = 12, 10, 16
    rmin, rmax = 0.3 * AU, 2.0 * AU
    dr, dth, dph = (rmax - rmin) / (nr - 1), np.pi / (nt - 1), 2 * np.pi / npf
    coef = RNG.normal(size=(4, 8))
    I, J, K = np.meshgrid(np.arange(nr), np.arange(nt), np.arange(npf), indexing="ij")
    nodes = np.empty((npf, nt, nr, 8))
    for ch in range(8):
        val = coef[0, ch] + coef[1, ch] * I + coef[2, ch] * J + coef[3, ch] * K
        nodes[:, :, :, ch] = np.transpose(val, (2, 1, 0))
    f = oracle.grid_field(nodes, rmin, rmax)

    def exact(X):
        xr, xt, xp = _coords(X, rmin, dr, dth, dph)
        return coef[0, :6] + coef[1, :6] * xr + coef[2, :6] * xt + coef[3, :6] * xp

    for _ in range(40):
        r = RNG.uniform(rmin + dr, rmax - dr)
        th = RNG.uniform(2 * dth, np.pi - 2 * dth)
        ph = RNG.uniform(0.3 * dph, 2 * np.pi - 1.3 * dph)  # stay off the periodic seam
        X = node_xyz(r, th, ph)
        out, fl = oracle.field_eval(f, X)
        assert fl == 0
        ex = exact(X)
        np.testing.assert_allclose(out["B"], ex[0:3], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(out["E"], ex[3:6], rtol=1e-10, atol=1e-10)
        h = 1e-6 * r
        fd = np.zeros((6, 3))
        for jx in range(3):
            e = np.zeros(3)
            e[jx] = h
            fd[:, jx] = (exact(X + e) - exact(X - e)) / (2 * h)
        scale = np.abs(fd).max()
        np.testing.assert_allclose(out["JB"], fd[0:3], atol=1e-6 * scale)
        np.testing.assert_allclose(out["JE"], fd[3:6], atol=1e-6 * scale)


def _parker_grid(n):
    spec = synth.WindSpec(n_r=4 * n, n_th=2 * n, n_ph=4 * n, r_min_au=0.2, r_max_au=2.2)
    return spec, synth.wind_grid(spec, dtype=np.float64)


def test_grid_converges_to_analytic_parker():
    """Interpolating the Parker wind (sampled by the input generator) converges to the
    oracle's analytic Parker field: O(h^2) for values, O(h) for Jacobians."""
    fa = oracle.analytic_field(parker_B0=3.5e-9, parker_rref=AU, parker_omega=2.7e-6,
                               parker_u=4e5, parker_E=True)
    pts = [node_xyz(RNG.uniform(0.4, 1.9) * AU, RNG.uniform(0.6, 2.5), RNG.uniform(0, 2 * np.pi))
           for _ in range(200)]
    errB, errJ = [], []
    for n in (8, 16, 32):
        spec, nodes = _parker_grid(n)
        fg = oracle.grid_field(nodes, spec.r_min_au * AU, spec.r_max_au * AU)
        eb, ej = [], []
        for X in pts:
            g, _ = oracle.field_eval(fg, X)
            a, _ = oracle.field_eval(fa, X)
            eb.append(np.linalg.norm(g["B"] - a["B"]) / np.linalg.norm(a["B"]))
            ej.append(np.abs(g["JB"] - a["JB"]).max() / np.abs(a["JB"]).max())
        # rms over points: the error coefficient depends on the position inside a cell
        errB.append(np.sqrt(np.mean(np.square(eb))))
        errJ.append(np.sqrt(np.mean(np.square(ej))))
    rb = np.log2(np.array(errB[:-1]) / np.array(errB[1:]))
    rj = np.log2(np.array(errJ[:-1]) / np.array(errJ[1:]))
    assert np.all(rb > 1.7), (errB, rb)
    assert np.all(rj > 0.8), (errJ, rj)
    assert errB[-1] < 1e-3


@pytest.mark.parametrize("what", ["parker", "dipole", "uniform+parker"])
def test_analytic_jacobians_match_finite_differences(what):
    kw = dict(parker_B0=0.0)
    if what == "parker":
        kw = dict(parker_B0=3.5e-9, parker_E=True)
    elif what == "dipole":
        kw = dict(dipole_m=(1e22, -2e21, 5e22))
    else:
        kw = dict(B_unif=(1e-9, 2e-9, -1e-9), E_unif=(1e-4, 0, 2e-4), parker_B0=-2e-9,
                  parker_E=True)
    f = oracle.analytic_field(**kw)
    for _ in range(20):
        X = node_xyz(RNG.uniform(0.3, 2) * AU, RNG.uniform(0.3, 2.8), RNG.uniform(0, 6.28))
        out, _ = oracle.field_eval(f, X)
        h = 1e-5 * np.linalg.norm(X)
        for key, J in (("B", "JB"), ("E", "JE")):
            fd = np.zeros((3, 3))
            for jx in range(3):
                e = np.zeros(3)
                e[jx] = h
                fp, _ = oracle.field_eval(f, X + e)
                fm, _ = oracle.field_eval(f, X - e)
                fd[:, jx] = (fp[key] - fm[key]) / (2 * h)
            scale = max(np.abs(fd).max(), 1e-300)
            np.testing.assert_allclose(out[J], fd, atol=1e-7 * scale + 1e-300)


def test_parker_vector_identities_and_textbook_form():
    u, om, B1 = 4e5, 2.7e-6, 3.5e-9
    f = oracle.analytic_field(parker_B0=B1, parker_omega=om, parker_u=u, parker_E=True)
    for _ in range(20):
        r, th, ph = RNG.uniform(0.2, 2.4) * AU, RNG.uniform(0.2, 2.9), RNG.uniform(0, 6.28)
        X = node_xyz(r, th, ph)
        out, _ = oracle.field_eval(f, X)
        B, E, JB, JE = out["B"], out["E"], out["JB"], out["JE"]
        rhat = X / r
        that = np.array([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
        phat = np.array([-np.sin(ph), np.cos(ph), 0.0])
        Br, Bt, Bp = B @ rhat, B @ that, B @ phat
        # textbook Parker spiral: B_r = B1 (1AU/r)^2, B_theta = 0, B_phi = -B_r Omega r sin / u
        np.testing.assert_allclose(Br, B1 * (AU / r) ** 2, rtol=1e-12)
        assert abs(Bt) < 1e-12 * abs(Br)
        np.testing.assert_allclose(Bp, -Br * om * r * np.sin(th) / u, rtol=1e-12)
        # ideal Ohm's law with a radial wind
        np.testing.assert_allclose(E, -np.cross(u * rhat, B), rtol=1e-12, atol=1e-20)
        assert abs(E @ B) < 1e-12 * np.linalg.norm(E) * np.linalg.norm(B)
        # E along -theta in the north for B_r > 0 (Eq. 14 discussion)
        if th < np.pi / 2:
            assert E @ that < 0
        assert abs(np.trace(JB)) < 1e-10 * np.abs(JB).max()
        curlE = np.array([JE[2, 1] - JE[1, 2], JE[0, 2] - JE[2, 0], JE[1, 0] - JE[0, 1]])
        assert np.abs(curlE).max() < 1e-10 * np.abs(JE).max()


def test_dipole_identities():
    m = np.array([0.0, 0.0, 8e22])
    f = oracle.analytic_field(dipole_m=tuple(m))
    r = 0.5 * AU
    out, _ = oracle.field_eval(f, np.array([r, 0, 0]))
    np.testing.assert_allclose(out["B"], -m / r**3, rtol=1e-13)
    for _ in range(10):
        X = node_xyz(RNG.uniform(0.3, 2) * AU, RNG.uniform(0.3, 2.8), RNG.uniform(0, 6.28))
        out, _ = oracle.field_eval(f, X)
        JB = out["JB"]
        assert abs(np.trace(JB)) < 1e-10 * np.abs(JB).max()
        curl = np.array([JB[2, 1] - JB[1, 2], JB[0, 2] - JB[2, 0], JB[1, 0] - JB[0, 1]])
        assert np.abs(curl).max() < 1e-10 * np.abs(JB).max()


def test_synth_perturbation_is_solenoidal_with_stated_amplitude():
    spec = synth.WindSpec(n_r=64, n_th=32, n_ph=64, eps=0.1, n_modes=8, seed=0)
    base = synth.WindSpec(n_r=64, n_th=32, n_ph=64)
    X = np.stack([node_xyz(RNG.uniform(0.3, 2.2) * AU, RNG.uniform(0.5, 2.6),
                           RNG.uniform(0, 6.28)) for _ in range(400)])
    B, _ = synth.wind_at(spec, X)
    B0, _ = synth.wind_at(base, X)
    rel = np.linalg.norm(B - B0, axis=1) / np.linalg.norm(B0, axis=1)
    assert 0.03 < np.sqrt(np.mean(rel**2)) < 0.3
    h = 1e-5 * AU
    div = np.zeros(len(X))
    for jx in range(3):
        e = np.zeros(3)
        e[jx] = h
        Bp, _ = synth.wind_at(spec, X + e)
        Bm, _ = synth.wind_at(spec, X - e)
        div += (Bp[:, jx] - Bm[:, jx]) / (2 * h)
    # |B| / (0.1 AU) is the size of a single derivative term
    scale = np.linalg.norm(B, axis=1) / (0.1 * AU)
    assert np.abs(div / scale).max() < 1e-5


def test_synth_grid_matches_wind_at_nodes():
    spec = synth.WindSpec(n_r=10, n_th=8, n_ph=12, eps=0.1, n_modes=4)
    g = synth.wind_grid(spec, dtype=np.float64)
    r, th, ph = grid_axes(10, 8, 12, spec.r_min_au * AU, spec.r_max_au * AU)
    X = node_xyz(r[3], th[2], ph[5])
    B, E = synth.wind_at(spec, X[None])
    np.testing.assert_allclose(g[5, 2, 3, 0:3], B[0], rtol=1e-12)
    np.testing.assert_allclose(g[5, 2, 3, 3:6], E[0], rtol=1e-12)
    np.testing.assert_allclose(g[5, 2, 3, 6], np.linalg.norm(B[0]), rtol=1e-12)


def test_synth_grid_is_the_same_on_any_number_of_threads():
    spec = synth.WindSpec(n_r=24, n_th=10, n_ph=20, eps=0.2, n_modes=6, phi1_v=500.0)
    serial = synth.wind_grid(spec, dtype=np.float64, workers=1)
    for w in (2, 7):
        np.testing.assert_array_equal(synth.wind_grid(spec, dtype=np.float64, workers=w), serial)

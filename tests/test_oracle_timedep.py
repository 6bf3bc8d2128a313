"""Time-dependent fields: two grid snapshots, every field quantity linear in time between
them (held constant outside), and the time-derivative terms of the guiding-centre equations
that vanish for the paper's steady wind (Eqs. 1-2 in the form of the GCA source the paper
cites, Sect. 2.2): v_par db/dt + dv_E/dt inside the bracket of Eq. 1 and gamma v_E . db/dt in
Eq. 2.

Pins: (1) the snapshot blend and its secant time derivative, and the clamp outside the
window; (2) the polarization drift gamma m (dE/dt) / (q B^2) of a uniform E growing across a
uniform B (the textbook closed form); (3) for uniform fields changing in magnitude and
direction, db/dt and dv_E/dt of the oracle against SymPy's time derivatives of b(t) and
v_E(t), through the whole right-hand side."""
import numpy as np
import sympy as sp

import oracle
from oracle import AU, C_LIGHT, M_E, Q_E
from paper_2403_06706_gb300 import synth

RNG = np.random.default_rng(21)
W = synth.WindSpec(32, 16, 32)


def _uniform(B, E):
    nodes = np.zeros((W.n_ph, W.n_th, W.n_r, 8))
    nodes[..., 0:3] = B
    nodes[..., 3:6] = E
    nodes[..., 6] = np.linalg.norm(B)
    return nodes


def _pair(n0, n1, T):
    return oracle.grid_field_pair(n0, n1, 0.0, T, W.r_min_au * AU, W.r_max_au * AU)


def _point():
    r = RNG.uniform(0.3, 2.0) * AU
    th = np.arccos(RNG.uniform(-0.9, 0.9))
    ph = RNG.uniform(0, 2 * np.pi)
    return r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


def test_snapshot_blend_secant_and_clamp():
    n0 = synth.wind_grid(W, dtype=np.float64)
    n1 = synth.wind_grid(synth.WindSpec(32, 16, 32, eps=0.2, n_modes=4, seed=3), dtype=np.float64)
    T = 3600.0
    fp = _pair(n0, n1, T)
    f0 = oracle.grid_field(n0, W.r_min_au * AU, W.r_max_au * AU)
    f1 = oracle.grid_field(n1, W.r_min_au * AU, W.r_max_au * AU)
    for _ in range(20):
        R = _point()
        t = RNG.uniform(0, T)
        a, _ = oracle.field_eval(f0, R)
        b, _ = oracle.field_eval(f1, R)
        s, _ = oracle.field_eval(fp, R, t)
        w = t / T
        for k in ("B", "E", "JB", "JE"):
            np.testing.assert_allclose(s[k], (1 - w) * a[k] + w * b[k], rtol=1e-12,
                                       atol=1e-15 * np.abs(a[k]).max())
        np.testing.assert_allclose(s["dBdt"], (b["B"] - a["B"]) / T, rtol=1e-12)
        np.testing.assert_allclose(s["dEdt"], (b["E"] - a["E"]) / T, rtol=1e-12)
        before, _ = oracle.field_eval(fp, R, -10.0)
        after, _ = oracle.field_eval(fp, R, T + 10.0)
        np.testing.assert_allclose(before["B"], a["B"], rtol=1e-14)
        np.testing.assert_allclose(after["B"], b["B"], rtol=1e-14)
        assert not before["dBdt"].any() and not after["dEdt"].any()


def test_polarization_drift_closed_form():
    B0, E0, T, grow = 5e-9, 2e-3, 1000.0, 0.5
    fp = _pair(_uniform([0, 0, B0], [E0, 0, 0]), _uniform([0, 0, B0], [E0 * (1 + grow), 0, 0]), T)
    p = oracle.params()
    for _ in range(5):
        R = _point()
        t = RNG.uniform(0.1, 0.9) * T
        mub = RNG.uniform(1e-17, 1e-16)
        u = RNG.uniform(-1e8, 1e8)
        F, aux, _ = oracle.rhs(fp, p, np.r_[R, u], mub, t)
        gam, vpar = aux[0], aux[1]
        E = E0 * (1 + grow * t / T)
        vE = np.array([0.0, -E / B0, 0.0])
        vpol = gam * M_E * (E0 * grow / T) / (Q_E * B0**2) * np.array([1.0, 0, 0])
        np.testing.assert_allclose(F[0:3] - vpar * np.array([0, 0, 1.0]) - vE, vpol, rtol=1e-10,
                                   atol=1e-12 * np.abs(vE).max())
        assert abs(F[3]) < 1e-12 * abs(u)


def _sympy_uniform_rhs(B0, Bdot, E0, Edot, q, m):
    t, u, mub = sp.symbols("t u mub", real=True)
    Bv = sp.Matrix(B0) + t * sp.Matrix(Bdot)
    Ev = sp.Matrix(E0) + t * sp.Matrix(Edot)
    Bm = sp.sqrt(Bv.dot(Bv))
    b = Bv / Bm
    vE = Ev.cross(b) / Bm
    c2 = C_LIGHT**2
    gam = sp.sqrt(1 + (u**2 + 2 * mub * Bm / m) / c2)
    vpar = u / gam
    # uniform fields: every spatial derivative vanishes; the time terms remain
    db = sp.diff(b, t)
    dvE = sp.diff(vE, t)
    br = vpar * db + dvE
    dR = vpar * b + vE + (gam * m / (q * Bm)) * b.cross(br)
    du = gam * vE.dot(db)
    return sp.lambdify((t, u, mub), list(dR) + [du], "numpy")


def test_time_terms_match_sympy():
    T = 2000.0
    B0 = np.array([1e-9, -2e-9, 4e-9])
    B1 = np.array([3e-9, 1e-9, 3e-9])
    E0 = np.array([1e-3, 2e-3, 0.5e-3])
    E1 = np.array([-1e-3, 3e-3, 1e-3])
    fp = _pair(_uniform(B0, E0), _uniform(B1, E1), T)
    p = oracle.params(q=Q_E, m=M_E)
    fs = _sympy_uniform_rhs(B0, (B1 - B0) / T, E0, (E1 - E0) / T, Q_E, M_E)
    for _ in range(6):
        R = _point()
        t = RNG.uniform(0.1, 0.9) * T
        mub = RNG.uniform(1e-17, 1e-16)
        u = RNG.uniform(-1e8, 1e8)
        F, _, _ = oracle.rhs(fp, p, np.r_[R, u], mub, t)
        ref = np.array(fs(t, u, mub), dtype=float)
        np.testing.assert_allclose(F[0:3], ref[0:3], rtol=1e-9, atol=1e-9 * np.abs(ref[0:3]).max())
        np.testing.assert_allclose(F[3], ref[3], rtol=1e-8, atol=1e-9 * abs(u))

"""The two-fluid electric field (Sect. 2.2): E = -u x B - grad(p)/(e n), and with p = p(n)
the correction is -grad(Phi). Ideal interpolated E carries no physical E_par, so in this
mode E_par = -b.grad(Phi) with Phi the grid's potential channel (its trilinear
interpolant's gradient).

Pins: (1) for a potential that depends on r only, the interpolant's gradient is radial and
equals the secant slope between the bracketing radial nodes, exactly; (2) with E = 0 apart
from the potential and only the v_par b motion kept, the guiding centre moves along b and
the energy (gamma - 1) m c^2 + q Phi(R) is conserved, while the kinetic energy itself changes
by -q dPhi (electrons running outward down the potential lose energy)."""
import numpy as np

import oracle
from _cases import oracle_ensembles
from oracle import AU, C_LIGHT, M_E, Q_E
from paper_2403_06706_gb300 import synth

RNG = np.random.default_rng(12)
W = synth.WindSpec(64, 32, 64, phi1_v=50.0, gamma_p=1.2)
W_STRONG = synth.WindSpec(64, 32, 64, phi1_v=500.0, gamma_p=1.2)


def test_potential_gradient_is_the_radial_secant_slope():
    nodes = synth.wind_grid(W, dtype=np.float64)
    f = oracle.grid_field(nodes, W.r_min_au * AU, W.r_max_au * AU, ideal=2)
    dr = W.dr_au * AU
    r_nodes = (W.r_min_au + W.dr_au * np.arange(W.n_r)) * AU
    phi = W.phi1_v * (AU / r_nodes) ** (2 * (W.gamma_p - 1))
    for _ in range(50):
        r = RNG.uniform(0.15, 2.4) * AU
        th = np.arccos(RNG.uniform(-0.9, 0.9))
        ph = RNG.uniform(0, 2 * np.pi)
        R = r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        s, _ = oracle.field_eval(f, R)
        i = int((r - W.r_min_au * AU) // dr)
        slope = (phi[i + 1] - phi[i]) / dr
        np.testing.assert_allclose(s["gPhi"], slope * R / r, rtol=1e-9, atol=1e-12 * abs(slope))


def test_energy_with_the_potential_is_conserved_along_b():
    # mu0 = 1 (mu_B = 0): no mirror force, whose jumps across the trilinear cells would
    # blur the energy budget; a 10x stronger potential for a clear signal
    W = W_STRONG
    nodes = synth.wind_grid(W, dtype=np.float64)
    nodes[..., 3:6] = 0.0  # no motional field: E = -grad(Phi) only
    f = oracle.grid_field(nodes, W.r_min_au * AU, W.r_max_au * AU, ideal=2)
    ens = (synth.EnsembleSpec(64, lam_au=0.5, r_out_au=2.4, mu_law=1),)
    p = oracle.params(seed=3, drift_mask=1, no_scatter=True, no_rebirth=True)
    oe = oracle_ensembles(ens)
    st = oracle.inject(f, p, oe, [64], dt=0.5)

    def energies(s):
        K, U = np.empty(s.n), np.empty(s.n)
        for i in range(s.n):
            R = np.array([s["x"][i], s["y"][i], s["z"][i]])
            fl, _ = oracle.field_eval(f, R)
            B = np.linalg.norm(fl["B"])
            g = np.sqrt(1 + (s["u"][i] ** 2 + 2 * s["mub"][i] * B / M_E) / C_LIGHT**2)
            # the potential at R: trilinear value of channel 7 along r
            r = np.linalg.norm(R)
            rn = (W.r_min_au + W.dr_au * np.arange(W.n_r)) * AU
            U[i] = Q_E * np.interp(r, rn, W.phi1_v * (AU / rn) ** (2 * (W.gamma_p - 1)))
            K[i] = (g - 1) * M_E * C_LIGHT**2
        return K, U

    K0, U0 = energies(st)
    oracle.advance(f, p, oe, st, 0.0, 0, 0.5, 480)
    K1, U1 = energies(st)
    dK = K1 - K0
    print("kinetic change (eV):", dK.mean() / 1.602176634e-19, "total change / kinetic change:",
          np.abs(dK + (U1 - U0)).max() / np.abs(dK).max())
    assert (dK < 0).all()                  # outward electrons climb into lower potential: q Phi rises
    assert np.abs(dK).max() > 1e-19        # the field does work (> 1 eV)
    assert np.abs(dK + (U1 - U0)).max() < 1e-3 * np.abs(dK).max()

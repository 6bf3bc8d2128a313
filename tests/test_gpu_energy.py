"""Energy bookkeeping of the FP32-mixed push across many collisions (Sect. 2.3: elastic
collisions in the inertial frame keep |p|; Sect. 3: the drift energy loss, ~10 % per day, is
the signal the FP64 bookkeeping exists to keep).

A uniform field B = (B0, 0, 0) with E = 0 and no gradient: between collisions every term of
Eq. 2 vanishes, so gamma changes only at collisions. B0 = 2^-28 T is exact in float, so the
kernel's |B| equals the host's. With lambda = 1e-4 AU most steps of an 81 keV electron end in
a collision (at most one per step; a particle left with |mu| near 0 travels little along B
and waits longer), ~6000 collisions per particle in 10^4 steps, under both scattering laws
(Eqs. 10 and 12).

Bound: a collision recomputes |p|^2 = (gamma v_par)^2 + 2 mu_B |B| / m in FP64 from the
double-float gamma v_par (48 significand bits) and the FP64 mu_B of the state, then stores
the new pair. Its relative error is at most 2^-47 (the double-float rounding, squared) plus
about eight FP64 roundings, < 1e-14; with (gamma^2 - 1) / (2 gamma^2) = 0.13 at 81 keV the
error of gamma after 10^4 collisions, even added up linearly, stays below 2e-11. The test
holds it to 1e-10, nearly three decades below one FP32 rounding (6e-8) per collision, the
level a float collision update leaves (~1e-6 after 10^4 collisions); the oracle's FP64 run of
the same particles is held to the same bound.
"""
import numpy as np
import pytest

import oracle
from oracle import AU, C_LIGHT, M_E
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")

B0 = 2.0 ** -28  # T


def _uniform_nodes(dtype):
    nodes = np.zeros((32, 16, 16, 8), dtype=dtype)
    nodes[..., 0] = B0
    nodes[..., 6] = B0
    return nodes


def _gamma(st):
    pm2 = st["u"] ** 2 + 2.0 * st["mub"] * B0 / M_E
    return np.sqrt(1.0 + pm2 / C_LIGHT ** 2)


def test_fp32_collisions_keep_gamma_to_fp64_rounding():
    ens = [synth.EnsembleSpec(count=1024, r0_au=1.0, lat_deg=0.0, lam_au=1e-4, r_in_au=0.5, r_out_au=2.0,
                              scatter_law=law) for law in (0, 1)]
    nodes = _uniform_nodes(np.float32)
    n_steps = 10000
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=3, dt_init=0.5) as c:
        c.field_load(nodes, 0.1, 2.5)
        c.inject(ens)
        g0 = c.get_state()
        for _ in range(4):
            c.advance(0.5, n_steps // 4)
        g1 = c.get_state()
        s = c.stats()
    assert int(s["rebirths"]) == 0
    assert int(s["collisions"]) >= 0.5 * 2048 * n_steps, s["collisions"]
    assert np.all(g1["flags"] == 0)
    dg = np.abs(_gamma(g1) / _gamma(g0) - 1.0)
    print("FP32 path: |gamma/gamma0 - 1| max", dg.max(), "rms", np.sqrt(np.mean(dg ** 2)))
    assert dg.max() < 1e-10

    # the FP64 oracle on the first 64 particles of each law
    f = oracle.grid_field(_uniform_nodes(np.float64), 0.1 * AU, 2.5 * AU)
    p = oracle.params(seed=3)
    oe = [oracle.ensemble(r0_au=1.0, lat_deg=0.0, lam_au=1e-4, r_in_au=0.5, r_out_au=2.0, scatter_law=law)
          for law in (0, 1)]
    st = oracle.inject(f, p, oe, [1024, 1024], dt=0.5)
    st = st.subset(np.r_[0:64, 1024:1088])
    o0 = {k: st[k].copy() for k in ("u", "mub")}
    oracle.advance(f, p, oe, st, 0.0, 0, 0.5, n_steps)
    do = np.abs(_gamma(st) / _gamma(o0) - 1.0)
    print("FP64 oracle: |gamma/gamma0 - 1| max", do.max())
    assert do.max() < 1e-10
    assert st["ncoll"].mean() >= 0.5 * n_steps

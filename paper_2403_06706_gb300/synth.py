"""Seeded synthetic inputs: the solar-wind field grid and the particle workloads.

This module is the only one shared by the CUDA path and the FP64 oracle. It
holds none of the transport method's arithmetic: it samples an input field on
the grid nodes and describes workloads. The paper propagates electrons in a
steady MPI-AMRVAC MHD wind (Sect. 2.1) that is not available here; the
stand-in is an analytic Parker spiral (the model the paper compares its wind
to, Sect. 2.1) plus a seeded, exactly divergence-free perturbation:

* Parker: u = u_sw rhat, B_r = B1 (1 AU / r)^2, B_phi = -B_r Omega r sin(theta) / u_sw
  (unipolar, B_r > 0: the polarity for which the paper's signs hold — the
  E x B drift to +phi, Sect. 3, and E along -theta, Eq. 14).
* perturbation: dB = curl(g(r) A), A = sum_m a_m e_m sin(k_m.x + psi_m) / |k_m|,
  e_m a random unit vector normal to k_m, directions uniform on the sphere,
  wavelengths log-spaced from 1 AU down to four angular cells at 1 AU,
  a_m ~ |k_m|^(-5/6) normalised so that sum a_m^2 / 2 = 1, and
  g(r) = eps B1 (1 AU / r)^2 sqrt(1 + (Omega r / u_sw)^2), so that the rms of
  dB/|B| is about eps. curl(g A) = g'(r) rhat x A + g curl A.
* ideal Ohm's law: E = -u x B at every node.
* optional two-fluid potential (channel Phi): a polytropic wind with n ~ 1/r^2 and
  p ~ n^G has -grad(p)/(e n) = -grad(Phi) with Phi = phi1 (1 AU / r)^(2 (G - 1)) (phi1: the
  potential at 1 AU, G = gamma_p); a few hundred volts between the corona and 1 AU.

Node records are 8 channels [Bx, By, Bz, Ex, Ey, Ez, |B|, Phi] (Cartesian
components, SI units), node-centred, laid out [i_phi][i_theta][i_r][channel]:
r_i = r_min + i dr, theta_j = j pi / (n_th - 1) (poles included),
phi_k = 2 pi k / n_ph (periodic). Phi (the two-fluid potential channel) is 0
unless phi1_v is set. All draws come from numpy's PCG64 with the given seed.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

AU = 1.495978707e11  # m
KEV = 1.602176634e-16  # J
R_SUN_DEG = np.pi / 180.0


@dataclass(frozen=True)
class WindSpec:
    n_r: int = 64
    n_th: int = 32
    n_ph: int = 64
    r_min_au: float = 0.1
    r_max_au: float = 2.5
    B1: float = 3.5e-9  # B_r at 1 AU, T
    omega: float = 2.7e-6  # solar rotation, rad/s
    u_sw: float = 4.0e5  # wind speed, m/s
    eps: float = 0.0  # rms dB/|B| of the perturbation
    n_modes: int = 0
    seed: int = 0
    phi1_v: float = 0.0  # two-fluid potential at 1 AU, V (0: none)
    gamma_p: float = 1.2  # polytropic index of the potential

    @property
    def dr_au(self) -> float:
        return (self.r_max_au - self.r_min_au) / (self.n_r - 1)


def perturbation_modes(spec: WindSpec):
    """Mode table (k [1/m] (n,3), e (n,3), psi (n,), a (n,)) of the perturbation."""
    n = spec.n_modes
    rng = np.random.default_rng(spec.seed)
    if n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0)
    l_max = 1.0 * AU
    l_min = 4.0 * (np.pi / (spec.n_th - 1)) * AU  # four angular cells at 1 AU
    ell = np.geomspace(l_max, l_min, n) if n > 1 else np.array([l_max])
    kmag = 2.0 * np.pi / ell
    # uniform directions on the sphere
    kz = rng.uniform(-1.0, 1.0, n)
    kp = rng.uniform(0.0, 2.0 * np.pi, n)
    khat = np.stack([np.sqrt(1 - kz**2) * np.cos(kp), np.sqrt(1 - kz**2) * np.sin(kp), kz], 1)
    # a random unit vector normal to k
    e = rng.normal(size=(n, 3))
    e -= (e * khat).sum(1, keepdims=True) * khat
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    psi = rng.uniform(0.0, 2.0 * np.pi, n)
    a = kmag ** (-5.0 / 6.0)
    a *= np.sqrt(2.0 / (a**2).sum())
    return khat * kmag[:, None], e, psi, a


def wind_at(spec: WindSpec, X: np.ndarray, modes=None) -> tuple[np.ndarray, np.ndarray]:
    """B and E (SI) of the synthetic wind at Cartesian points X (..., 3) in m."""
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    rhat = X / r[..., None]
    r1 = AU
    w = spec.omega / spec.u_sw
    # Parker: B = B1 r1^2 [R / r^3 - w (zhat x R) / r^2]
    zxR = np.stack([-y, x, np.zeros_like(z)], -1)
    C = spec.B1 * r1 * r1
    B = C * (X / (r**3)[..., None] - w * zxR / (r**2)[..., None])
    if spec.n_modes > 0:
        if modes is None:
            modes = perturbation_modes(spec)
        k, e, psi, a = modes
        s = np.sqrt(1.0 + (w * r) ** 2)
        g = spec.eps * C * s / r**2
        dg = spec.eps * C * (-2.0 * s / r**3 + w * w / (r * s))
        A = np.zeros_like(X)
        curlA = np.zeros_like(X)
        khat = k / np.linalg.norm(k, axis=1, keepdims=True)
        kxe = np.cross(khat, e)
        kmag = np.linalg.norm(k, axis=1)
        for m in range(k.shape[0]):
            ph = X @ k[m] + psi[m]
            A += (a[m] * np.sin(ph) / kmag[m])[..., None] * e[m]
            curlA += (a[m] * np.cos(ph))[..., None] * kxe[m]
        B = B + dg[..., None] * np.cross(rhat, A) + g[..., None] * curlA
    u = spec.u_sw * rhat
    E = -np.cross(u, B)
    return B, E


def potential_of(spec: WindSpec, phi1_v: float, gamma_p: float = 1.2) -> np.ndarray:
    """The polytropic potential channel (see module doc) on the radial nodes, shape (n_r,)."""
    r = (spec.r_min_au + spec.dr_au * np.arange(spec.n_r)) * AU
    return phi1_v * (AU / r) ** (2.0 * (gamma_p - 1.0))


def wind_grid(spec: WindSpec, dtype=np.float32, workers: int | None = None) -> np.ndarray:
    """Node array [n_ph][n_th][n_r][8] of the synthetic wind (see module doc). The phi slabs
    are independent and computed on `workers` threads (default: the host's cores, at most
    16); every slab runs the same arithmetic, so the array does not depend on the count."""
    r = (spec.r_min_au + spec.dr_au * np.arange(spec.n_r)) * AU
    th = np.pi * np.arange(spec.n_th) / (spec.n_th - 1)
    ph = 2.0 * np.pi * np.arange(spec.n_ph) / spec.n_ph
    modes = perturbation_modes(spec)
    out = np.empty((spec.n_ph, spec.n_th, spec.n_r, 8), dtype=dtype)
    T, Rr = np.meshgrid(th, r, indexing="ij")  # (n_th, n_r)

    def slab(k):
        X = np.stack([Rr * np.sin(T) * np.cos(ph[k]), Rr * np.sin(T) * np.sin(ph[k]),
                      Rr * np.cos(T)], -1)
        # exact poles: sin(pi) is not 0 in floating point
        X[0, :, 0:2] = 0.0
        X[-1, :, 0:2] = 0.0
        B, E = wind_at(spec, X, modes)
        out[k, :, :, 0:3] = B
        out[k, :, :, 3:6] = E
        out[k, :, :, 6] = np.sqrt((B * B).sum(-1))
        if spec.phi1_v != 0.0:
            out[k, :, :, 7] = spec.phi1_v * (AU / Rr) ** (2.0 * (spec.gamma_p - 1.0))
        else:
            out[k, :, :, 7] = 0.0

    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    if workers <= 1:
        for k in range(spec.n_ph):
            slab(k)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(slab, range(spec.n_ph)))
    return out


@dataclass(frozen=True)
class EnsembleSpec:
    """One ensemble of electrons (units: AU, keV, degrees)."""
    count: int
    r0_au: float = 0.28
    lat_deg: float = 24.0
    lon_deg: float = 0.0
    E0_keV: float = 81.0
    lam_au: float = 0.5
    r_in_au: float | None = None  # default: the injection radius
    r_out_au: float = 2.4
    energy_law: int = 0  # 0 mono-energetic, 1 power law on [E_lo, E_hi]
    E_lo_keV: float = 20.0
    E_hi_keV: float = 500.0
    E_index: float = 3.0
    mu_law: int = 0  # 0: mu0 uniform on (0, 1]; 1: mu0 = 1 (alpha = 0)
    scatter_law: int = 0  # 0: mu = 1 - 2a; 1: mu = +-sqrt(a)

    @property
    def r_in(self) -> float:
        return self.r0_au if self.r_in_au is None else self.r_in_au


@dataclass(frozen=True)
class Workload:
    name: str
    wind: WindSpec
    ensembles: tuple
    dt: float = 0.5
    n_steps: int = 3600
    grid_dtype: str = "f32"
    seed: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_particles(self) -> int:
        return int(sum(e.count for e in self.ensembles))


def r_out_default(w: WindSpec) -> float:
    """Outer shell radius: one radial cell inside the grid edge."""
    return w.r_max_au - w.dr_au


def c1_plain_fp64() -> Workload:
    """4096 electrons, 81 keV, r = 0.28 AU, 24 deg, lon 0, mu0 ~ U(0,1], Parker 64x32x64
    FP64, lambda = 0.5 AU, dt = 0.5 s, 30 min (3600 steps), seed 0."""
    w = WindSpec(64, 32, 64)
    e = EnsembleSpec(4096, lam_au=0.5, r_out_au=r_out_default(w))
    return Workload("parker64x32x64_fp64_4096e_30min", w, (e,), 0.5, 3600, "f64")


def c2_perturbed(n_per_lambda: int = 1_000_000, lambdas=(0.1, 0.5, 1.0)) -> Workload:
    """Parker + perturbation (eps 0.1, 8 modes) on 256x128x256 FP32; 81 keV electrons, one
    ensemble per lambda in {0.1, 0.5, 1.0} AU, 48 h simulated (345600 steps)."""
    w = WindSpec(256, 128, 256, eps=0.1, n_modes=8)
    ens = tuple(EnsembleSpec(n_per_lambda, lam_au=l, r_out_au=r_out_default(w)) for l in lambdas)
    return Workload("parker256x128x256_eps0.1_8modes_3x1e6e", w, ens, 0.5, 345600, "f32")


def c3_batched(seed: int = 0) -> Workload:
    """64 ensembles of uneven size floor(10^U(3,5)), energies log-U(10,300) keV, lambda
    log-U(0.05,2) AU, r0 U(0.1,0.5) AU, latitude U(-60,60) deg, lon 0, on C2's field; 24 h."""
    w = WindSpec(256, 128, 256, eps=0.1, n_modes=8)
    rng = np.random.default_rng(seed + 3)
    ens = []
    for _ in range(64):
        cnt = int(np.floor(10 ** rng.uniform(3, 5)))
        E0 = float(np.exp(rng.uniform(np.log(10), np.log(300))))
        lam = float(np.exp(rng.uniform(np.log(0.05), np.log(2.0))))
        r0 = float(rng.uniform(0.1 + w.dr_au, 0.5))
        lat = float(rng.uniform(-60, 60))
        ens.append(EnsembleSpec(cnt, r0_au=r0, lat_deg=lat, E0_keV=E0, lam_au=lam,
                                r_out_au=r_out_default(w)))
    return Workload("batched64_parker256x128x256", w, tuple(ens), 0.5, 172800, "f32")


def c5_large(n: int = 30_000_000) -> Workload:
    """512x256x512 FP32 grid, eps 0.2, 16 modes; 3e7 electrons, E^-3 on [20,500] keV,
    lambda = 0.3 AU, 96 h simulated."""
    w = WindSpec(512, 256, 512, eps=0.2, n_modes=16)
    e = EnsembleSpec(n, lam_au=0.3, energy_law=1, E_lo_keV=20, E_hi_keV=500, E_index=3.0,
                     r_out_au=r_out_default(w))
    return Workload("parker512x256x512_eps0.2_16modes_3e7e", w, (e,), 0.5, 691200, "f32")


# --------------------------------------------------------------------------------------
# Neural-field inputs: the network's initial weights (seeded draws of the method, handed to
# both the CUDA path and the oracle) and the scaling that makes the targets O(1).

SIREN_HIDDEN = 256
SIREN_OMEGA0 = 30.0


def siren_init(seed: int = 0, n_h: int = SIREN_HIDDEN, n_out: int = 8, omega0: float = SIREN_OMEGA0):
    """Flat float32 parameters in the order W1 (n_h x 3), b1, W2..W4 (n_h x n_h), b2..b4,
    W5 (n_out x n_h), b5, initialised as in Sitzmann et al. (2020): first layer
    U(-1/3, 1/3) (fan-in 3, its sine carries the frequency omega0); hidden layers with the
    frequency folded in, U(-sqrt(6/n_h), sqrt(6/n_h)); linear output layer
    U(-sqrt(6/n_h)/omega0, sqrt(6/n_h)/omega0); biases U(-1/sqrt(fan_in), 1/sqrt(fan_in))."""
    rng = np.random.default_rng(seed + 1000)
    parts = [rng.uniform(-1.0 / 3.0, 1.0 / 3.0, (n_h, 3)), rng.uniform(-1 / np.sqrt(3), 1 / np.sqrt(3), n_h)]
    lim = np.sqrt(6.0 / n_h)
    for _ in range(3):
        parts += [rng.uniform(-lim, lim, (n_h, n_h)), rng.uniform(-1 / np.sqrt(n_h), 1 / np.sqrt(n_h), n_h)]
    parts += [rng.uniform(-lim / omega0, lim / omega0, (n_out, n_h)),
              rng.uniform(-1 / np.sqrt(n_h), 1 / np.sqrt(n_h), n_out)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def field_scales(w: WindSpec) -> dict:
    """Scaling of the network's inputs and outputs: x = R / r_max; outputs are
    B (r / 1 AU)^2 / B1, E (r / 1 AU) / (B1 u_sw), |B| (r / 1 AU)^2 / B1 and Phi / (B1 u_sw AU)."""
    return {"r_scale": w.r_max_au * AU, "B_scale": w.B1, "E_scale": w.B1 * w.u_sw}


def siren_samples(n: int, w: WindSpec, seed: int = 0) -> np.ndarray:
    """n training points uniform in the volume of the grid's shell r_min <= r <= r_max,
    scaled by r_max (x = R / r_max), float32 (n, 3)."""
    rng = np.random.default_rng(seed + 2000)
    a, b = w.r_min_au**3, w.r_max_au**3
    r = (a + rng.uniform(0.0, 1.0, n) * (b - a)) ** (1.0 / 3.0) / w.r_max_au
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return (v * r[:, None]).astype(np.float32)


def c4_neural(n: int = 10_000_000) -> Workload:
    """The perturbed Parker field of c2_perturbed replaced by a SIREN trained on 10^7
    uniform-in-volume samples of its grid interpolant; n electrons at 81 keV, lambda 0.5 AU."""
    w = WindSpec(256, 128, 256, eps=0.1, n_modes=8)
    e = EnsembleSpec(n, lam_au=0.5, r_out_au=r_out_default(w))
    return Workload("siren_parker256x128x256_eps0.1_8modes_1e7e", w, (e,), 0.5, 172800, "f32",
                    extra={"n_samples": 10_000_000, "epochs": 50, "batch": 65536, "lr": 4e-4,
                           # Adam's step halved after 20, 30 and 40 epochs
                           "schedule": ((20, 4e-4), (10, 2e-4), (10, 1e-4), (10, 5e-5)),
                           "omega0": SIREN_OMEGA0})

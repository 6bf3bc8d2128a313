"""FP64 CPU oracle of the guiding-centre electron transport method (arXiv:2403.06706).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library of
``paper_2403_06706_gb300`` never imports, links or calls it, and the two share
no code; the only thing both sides consume is the seeded input generator
(``paper_2403_06706_gb300.synth``), which holds none of the method's
arithmetic.

The arithmetic lives in ``gc_oracle.c`` (plain C11, FP64, OpenMP over
particles, ``-ffp-contract=off``). This module only builds it with gcc and
marshals numpy arrays through ctypes. Each C function cites the passage of the
paper it follows:

* field evaluation: trilinear interpolation (Sect. 2.2) or analytic fields;
* right-hand side: Eqs. 1-3;
* predictor / corrector: Eqs. 5-6 and the backward-Euler start-up (Sect. 2.2);
* scattering: Eq. 9 (collision probability), Eq. 10 and Eq. 12 (post-collision
  laws), Sect. 2.3; rebirth, snapshots and tallies: Sect. 3;
* Philox-4x32-10 (Salmon et al. 2011) for every random draw.

Pins (tests/test_oracle_*.py) tie each of these to what the paper and the
mathematics fix. Parity of the tally energy trend in a Parker field is
unpinned: the paper's magnitudes come from an MHD wind that is not available.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

C_LIGHT = 299792458.0
M_E = 9.1093837015e-31
Q_E = -1.602176634e-19
AU = 1.495978707e11
KEV = 1.602176634e-16

FLAG_OUT_OF_GRID = 1
FLAG_AXIS = 2
FLAG_NONFINITE = 4


def build(force: bool = False) -> str:
    """Compile gc_oracle.c into liboracle.so next to it (gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Field(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("ideal", C.c_int32), ("dtype", C.c_int32),
        ("n_r", C.c_int32), ("n_th", C.c_int32), ("n_ph", C.c_int32),
        ("parker_E", C.c_int32), ("pad0", C.c_int32),
        ("nodes", C.c_void_p),
        ("r_min", C.c_double), ("r_max", C.c_double),
        ("B_unif", C.c_double * 3), ("E_unif", C.c_double * 3),
        ("parker_B0", C.c_double), ("parker_rref", C.c_double),
        ("parker_omega", C.c_double), ("parker_u", C.c_double),
        ("dipole_m", C.c_double * 3),
        ("siren", C.c_void_p), ("siren_omega0", C.c_double), ("siren_rscale", C.c_double),
        ("siren_Bs", C.c_double), ("siren_Es", C.c_double), ("siren_bf16", C.c_int32),
        ("pad1", C.c_int32), ("nodes1", C.c_void_p), ("t_snap0", C.c_double), ("t_snap1", C.c_double),
    ]


class Params(C.Structure):
    _fields_ = [
        ("q", C.c_double), ("m", C.c_double), ("seed", C.c_uint32),
        ("collision_form", C.c_int32), ("drift_mask", C.c_int32),
        ("no_scatter", C.c_int32), ("no_rebirth", C.c_int32), ("pad0", C.c_int32),
        ("wind_u", C.c_double),
    ]


class Ensemble(C.Structure):
    _fields_ = [
        ("r0", C.c_double), ("lat", C.c_double), ("lon", C.c_double),
        ("E0", C.c_double), ("E_lo", C.c_double), ("E_hi", C.c_double), ("E_index", C.c_double),
        ("lam", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
        ("energy_law", C.c_int32), ("mu_law", C.c_int32), ("scatter_law", C.c_int32),
        ("pad0", C.c_int32),
    ]


_DP = C.POINTER(C.c_double)
_UP = C.POINTER(C.c_uint32)
_U64P = C.POINTER(C.c_uint64)


class State(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("x", _DP), ("y", _DP), ("z", _DP), ("u", _DP), ("mub", _DP),
        ("F0", _DP), ("F1", _DP), ("vpar", _DP), ("s_rem", _DP), ("h_prev", _DP),
        ("t_birth", _DP), ("u_inj", _DP), ("mub_inj", _DP),
        ("id", _UP), ("ens", _UP), ("event", _UP), ("ncoll", _UP), ("flags", _UP),
    ]


class Tally(C.Structure):
    _fields_ = [
        ("cadence", C.c_int32), ("n_mu", C.c_int32), ("n_E", C.c_int32), ("n_r", C.c_int32),
        ("n_age", C.c_int32), ("n_ens", C.c_int32),
        ("t_start", C.c_double), ("E_lo", C.c_double), ("E_hi", C.c_double),
        ("r_lo", C.c_double), ("r_hi", C.c_double), ("age_max", C.c_double),
        ("rwin_lo", C.c_double), ("rwin_hi", C.c_double), ("age_young", C.c_double),
        ("h_mer", _UP), ("h_age", _UP), ("h_pad", _UP),
        ("m_cnt", _U64P), ("m_sin2", _U64P), ("n_seen", _U64P),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_philox4x32_10.argtypes = [_UP, _UP, _UP]
        L.orc_philox4x32_10.restype = None
        L.orc_u53.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_u53.restype = C.c_double
        L.orc_field_eval.argtypes = [C.POINTER(Field), _DP, C.c_double, _DP]
        L.orc_field_eval.restype = C.c_uint32
        L.orc_rhs.argtypes = [C.POINTER(Field), C.POINTER(Params), _DP, C.c_double, C.c_double, _DP, _DP]
        L.orc_rhs.restype = C.c_uint32
        L.orc_predictor.argtypes = [_DP, _DP, _DP, C.c_double, C.c_double, _DP]
        L.orc_corrector.argtypes = [_DP, _DP, _DP, _DP, C.c_double, C.c_double, _DP]
        L.orc_inject.argtypes = [C.POINTER(Field), C.POINTER(Params), C.POINTER(Ensemble), C.c_int,
                                 C.POINTER(C.c_int64), C.POINTER(State), C.c_uint32, C.c_double,
                                 C.c_double, C.c_int]
        L.orc_inject.restype = C.c_int
        L.orc_advance.argtypes = [C.POINTER(Field), C.POINTER(Params), C.POINTER(Ensemble), C.c_int,
                                  C.POINTER(State), C.c_double, C.c_int64, C.c_double, C.c_int64,
                                  C.c_double, C.POINTER(Tally), _U64P, C.c_int]
        L.orc_advance.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _up(a):
    return a.ctypes.data_as(_UP)


# --------------------------------------------------------------------------- #
# Philox and uniform helpers


def philox(ctr, key) -> np.ndarray:
    """Philox-4x32-10 block for counter ``ctr`` (4 words) and key ``key`` (2 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_up(c), _up(k), _up(o))
    return o


def u53(w_hi: int, w_lo: int) -> float:
    return lib().orc_u53(int(w_hi), int(w_lo))


# --------------------------------------------------------------------------- #
# Fields


def grid_field(nodes: np.ndarray, r_min: float, r_max: float, ideal=True) -> Field:
    """Grid field over node array [n_ph][n_th][n_r][8] (float64 or float32), radii in m.
    ideal: True (E_par = 0), False (E_par = E.b) or 2 (two-fluid: E_par = -b.grad(Phi))."""
    assert nodes.ndim == 4 and nodes.shape[3] == 8 and nodes.flags.c_contiguous
    f = Field()
    f.kind = 0
    f.ideal = 2 if ideal == 2 else (1 if ideal else 0)
    f.dtype = 0 if nodes.dtype == np.float64 else 1
    assert nodes.dtype in (np.float64, np.float32)
    f.n_ph, f.n_th, f.n_r = nodes.shape[0], nodes.shape[1], nodes.shape[2]
    f.nodes = nodes.ctypes.data
    f.r_min, f.r_max = r_min, r_max
    f._keep = nodes  # keep the array alive with the struct
    return f


def analytic_field(B_unif=(0, 0, 0), E_unif=(0, 0, 0), parker_B0=0.0, parker_rref=AU,
                   parker_omega=2.7e-6, parker_u=4.0e5, parker_E=True, dipole_m=(0, 0, 0),
                   ideal: bool = True) -> Field:
    f = Field()
    f.kind = 1
    f.ideal = 1 if ideal else 0
    f.B_unif[:] = list(B_unif)
    f.E_unif[:] = list(E_unif)
    f.parker_B0, f.parker_rref = parker_B0, parker_rref
    f.parker_omega, f.parker_u = parker_omega, parker_u
    f.parker_E = 1 if parker_E else 0
    f.dipole_m[:] = list(dipole_m)
    return f


def siren_field(params_flat, omega0: float, r_scale: float, B_scale: float, E_scale: float,
                bf16: bool = False, ideal: bool = True) -> Field:
    """Neural field (SIREN, oracle/siren.py layout): x = R / r_scale, B = B_scale y_B (AU/r)^2,
    E = E_scale y_E (AU/r). With bf16 the weights W2..W5 are rounded to bfloat16 here and the
    values carried between layers inside the evaluation (the tensor-core arithmetic)."""
    from . import siren as _siren
    P = np.ascontiguousarray(params_flat, dtype=np.float64).copy()
    if bf16:
        for k in range(2, 6):
            o = _siren.offset(f"W{k}")
            n = 65536 if k < 5 else 2048
            P[o:o + n] = _siren.round_bf16(P[o:o + n])
    f = Field()
    f.kind = 2
    f.ideal = 2 if ideal == 2 else (1 if ideal else 0)
    f.siren = P.ctypes.data
    f.siren_omega0, f.siren_rscale, f.siren_Bs, f.siren_Es = omega0, r_scale, B_scale, E_scale
    f.siren_bf16 = 1 if bf16 else 0
    f._keep = P
    return f


def params(seed: int = 0, q: float = Q_E, m: float = M_E, collision_form: int = 0,
           drift_mask: int = 0, no_scatter: bool = False, no_rebirth: bool = False,
           wind_u: float = 0.0) -> Params:
    """wind_u > 0: collisions in the frame of a radial wind of that speed (m/s), Sect. 3.2."""
    p = Params()
    p.q, p.m, p.seed = q, m, seed
    p.collision_form, p.drift_mask = collision_form, drift_mask
    p.no_scatter, p.no_rebirth = int(no_scatter), int(no_rebirth)
    p.wind_u = wind_u
    return p


def field_eval(f: Field, R, t: float = 0.0) -> tuple[dict, int]:
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(33)
    fl = lib().orc_field_eval(C.byref(f), _dp(R), float(t), _dp(out))
    return {"B": out[0:3], "E": out[3:6], "JB": out[6:15].reshape(3, 3),
            "JE": out[15:24].reshape(3, 3), "gPhi": out[24:27], "dBdt": out[27:30],
            "dEdt": out[30:33]}, fl


def rhs(f: Field, p: Params, X, mub: float, t: float = 0.0):
    """F(X, t) of Eqs. 1-2 and (gamma, v_par, |B|, E_par)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    F = np.zeros(4)
    aux = np.zeros(4)
    fl = lib().orc_rhs(C.byref(f), C.byref(p), _dp(X), float(t), float(mub), _dp(F), _dp(aux))
    return F, aux, fl


def grid_field_pair(nodes0: np.ndarray, nodes1: np.ndarray, t0: float, t1: float, r_min: float, r_max: float,
                    ideal=True) -> Field:
    """Two grid snapshots at times t0 < t1 (s): the field is linear in time between them and
    held outside."""
    assert nodes1.shape == nodes0.shape and nodes1.dtype == nodes0.dtype and nodes1.flags.c_contiguous
    assert t1 > t0
    f = grid_field(nodes0, r_min, r_max, ideal)
    f.nodes1 = nodes1.ctypes.data
    f.t_snap0, f.t_snap1 = t0, t1
    f._keep1 = nodes1
    return f


def predictor(X, F0, F1, dt, tau):
    X, F0, F1 = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, F0, F1))
    out = np.zeros(4)
    lib().orc_predictor(_dp(X), _dp(F0), _dp(F1), dt, tau, _dp(out))
    return out


def corrector(X, F0, F1, Fs, dt, tau):
    X, F0, F1, Fs = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, F0, F1, Fs))
    out = np.zeros(4)
    lib().orc_corrector(_dp(X), _dp(F0), _dp(F1), _dp(Fs), dt, tau, _dp(out))
    return out


# --------------------------------------------------------------------------- #
# Ensembles, state and tallies


def ensemble(r0_au=0.28, lat_deg=24.0, lon_deg=0.0, E0_keV=81.0, lam_au=0.5, r_in_au=None,
             r_out_au=2.4, energy_law=0, E_lo_keV=20.0, E_hi_keV=500.0, E_index=3.0,
             mu_law=0, scatter_law=0) -> Ensemble:
    e = Ensemble()
    e.r0 = r0_au * AU
    e.lat = np.deg2rad(lat_deg)
    e.lon = np.deg2rad(lon_deg)
    e.E0 = E0_keV * KEV
    e.E_lo, e.E_hi, e.E_index = E_lo_keV * KEV, E_hi_keV * KEV, E_index
    e.lam = lam_au * AU
    e.r_in = (r0_au if r_in_au is None else r_in_au) * AU
    e.r_out = r_out_au * AU
    e.energy_law, e.mu_law, e.scatter_law = energy_law, mu_law, scatter_law
    return e


STATE_F64 = ("x", "y", "z", "u", "mub", "vpar", "s_rem", "h_prev", "t_birth", "u_inj", "mub_inj")
STATE_U32 = ("id", "ens", "event", "ncoll", "flags")


@dataclass
class StateArrays:
    """Structure-of-arrays particle state (SI units); F0/F1 are [4][n]."""
    arrays: dict

    @classmethod
    def empty(cls, n: int) -> "StateArrays":
        a = {k: np.zeros(n) for k in STATE_F64}
        a.update({k: np.zeros(n, dtype=np.uint32) for k in STATE_U32})
        a["F0"] = np.zeros((4, n))
        a["F1"] = np.zeros((4, n))
        return cls(a)

    @property
    def n(self) -> int:
        return self.arrays["x"].shape[0]

    def __getitem__(self, k):
        return self.arrays[k]

    def copy(self) -> "StateArrays":
        return StateArrays({k: v.copy() for k, v in self.arrays.items()})

    def subset(self, idx) -> "StateArrays":
        out = {}
        for k, v in self.arrays.items():
            out[k] = np.ascontiguousarray(v[:, idx] if v.ndim == 2 else v[idx])
        return StateArrays(out)

    def cstruct(self) -> State:
        s = State()
        s.n = self.n
        for k in STATE_F64 + ("F0", "F1"):
            arr = self.arrays[k]
            assert arr.dtype == np.float64 and arr.flags.c_contiguous
            setattr(s, k, _dp(arr))
        for k in STATE_U32:
            arr = self.arrays[k]
            assert arr.dtype == np.uint32 and arr.flags.c_contiguous
            setattr(s, k, _up(arr))
        return s


def inject(f: Field, p: Params, ensembles, counts, id0=0, t0=0.0, dt=0.5,
           n_threads=0) -> StateArrays:
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    n = int(counts.sum())
    st = StateArrays.empty(n)
    earr = (Ensemble * len(ensembles))(*ensembles)
    cs = st.cstruct()
    rc = lib().orc_inject(C.byref(f), C.byref(p), earr, len(ensembles),
                          counts.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(cs), id0, t0, dt,
                          n_threads)
    if rc != 0:
        raise RuntimeError(f"orc_inject failed: {rc}")
    return st


@dataclass
class TallySpec:
    cadence: int = 100
    n_mu: int = 32
    n_E: int = 32
    n_r: int = 64
    n_age: int = 32
    t_start: float = 0.0
    E_lo_keV: float = 5.0
    E_hi_keV: float = 600.0
    r_lo_au: float = 0.1
    r_hi_au: float = 2.5
    age_max_s: float = 24 * 3600.0
    rwin_lo_au: float = 0.9
    rwin_hi_au: float = 1.1
    age_young_s: float = 1200.0


class TallyArrays:
    def __init__(self, spec: TallySpec, n_ens: int):
        self.spec = spec
        self.n_ens = n_ens
        self.h_mer = np.zeros((n_ens, spec.n_mu, spec.n_E, spec.n_r), dtype=np.uint32)
        self.h_age = np.zeros((n_ens, spec.n_age, spec.n_E), dtype=np.uint32)
        self.h_pad = np.zeros((n_ens, spec.n_mu), dtype=np.uint32)
        self.m_cnt = np.zeros((n_ens, spec.n_r), dtype=np.uint64)
        self.m_sin2 = np.zeros((n_ens, spec.n_r), dtype=np.uint64)
        self.n_seen = np.zeros(2, dtype=np.uint64)

    def cstruct(self) -> Tally:
        s = self.spec
        t = Tally()
        t.cadence, t.n_mu, t.n_E, t.n_r, t.n_age, t.n_ens = (s.cadence, s.n_mu, s.n_E, s.n_r,
                                                             s.n_age, self.n_ens)
        t.t_start = s.t_start
        t.E_lo, t.E_hi = s.E_lo_keV * KEV, s.E_hi_keV * KEV
        t.r_lo, t.r_hi = s.r_lo_au * AU, s.r_hi_au * AU
        t.age_max = s.age_max_s
        t.rwin_lo, t.rwin_hi = s.rwin_lo_au * AU, s.rwin_hi_au * AU
        t.age_young = s.age_young_s
        t.h_mer, t.h_age, t.h_pad = _up(self.h_mer), _up(self.h_age), _up(self.h_pad)
        t.m_cnt = self.m_cnt.ctypes.data_as(_U64P)
        t.m_sin2 = self.m_sin2.ctypes.data_as(_U64P)
        t.n_seen = self.n_seen.ctypes.data_as(_U64P)
        return t


def advance(f: Field, p: Params, ensembles, st: StateArrays, t0: float, step0: int, dt: float,
            n_steps: int, lambda_override_m: float = 0.0, tally: TallyArrays | None = None,
            n_threads: int = 0) -> np.ndarray:
    """Advance ``st`` in place; returns [collisions, rebirths]."""
    earr = (Ensemble * len(ensembles))(*ensembles)
    cs = st.cstruct()
    stats = np.zeros(2, dtype=np.uint64)
    tp = C.byref(tally.cstruct()) if tally is not None else None
    rc = lib().orc_advance(C.byref(f), C.byref(p), earr, len(ensembles), C.byref(cs), t0, step0,
                           dt, n_steps, lambda_override_m, tp, stats.ctypes.data_as(_U64P),
                           n_threads)
    if rc != 0:
        raise RuntimeError(f"orc_advance failed: {rc}")
    return stats

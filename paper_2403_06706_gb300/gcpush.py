"""Thin ctypes binding of libgcpush (C ABI declared in include/gcpush.h).

Argument marshalling only: every step of the transport method runs in the CUDA kernels
of ``csrc/``. The library is built in-tree by :func:`build` (nvcc, sm_103a); if it is
missing, :func:`load` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .synth import AU, KEV, EnsembleSpec

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
LIB_PATH = os.path.join(_HERE, "libgcpush.so")
SOURCES = ("gc_api.cu", "gc_push.cu", "gc_sort.cu", "gc_noalloc.cu", "gc_siren.cu", "gc_siren_eval.cu",
           "gc_neural.cu", "gc_peak.cu")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + _INCLUDE]

GC_OK = 0
GC_ERR = {-1: "GC_ERR_INVALID", -2: "GC_ERR_CUDA", -3: "GC_ERR_NOMEM", -4: "GC_ERR_STATE",
          -5: "GC_ERR_DEVICE_ANOMALY", -6: "GC_ERR_UNSUPPORTED"}
PREC_FP64, PREC_FP32_MIXED = 0, 1
DTYPE_F64, DTYPE_F32 = 0, 1


def _nvcc() -> str:
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.isabs(p) and os.path.exists(p) or not os.path.isabs(p)):
            return p
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (one TU per thread) and link libgcpush.so in-tree."""
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, h) for h in os.listdir(_CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(_INCLUDE, "gcpush.h"))
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return LIB_PATH
    objdir = os.path.join(_HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
                        *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# --------------------------------------------------------------------------- #
# C structures (mirror include/gcpush.h)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p),
                ("seed", C.c_uint32), ("collision_form", C.c_int32), ("drift_mask", C.c_int32),
                ("no_scatter", C.c_int32), ("no_rebirth", C.c_int32), ("id_base", C.c_uint32),
                ("charge", C.c_double), ("mass", C.c_double), ("dt_init", C.c_double),
                ("wind_u", C.c_double)]


class GridDesc(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_th", C.c_int32), ("n_ph", C.c_int32), ("dtype", C.c_int32),
                ("r_min_au", C.c_double), ("r_max_au", C.c_double), ("ideal", C.c_int32),
                ("pad0", C.c_int32)]


class EnsembleDesc(C.Structure):
    _fields_ = [("count", C.c_int64), ("r0_au", C.c_double), ("lat_deg", C.c_double),
                ("lon_deg", C.c_double), ("E0_keV", C.c_double), ("E_lo_keV", C.c_double),
                ("E_hi_keV", C.c_double), ("E_index", C.c_double), ("lambda_au", C.c_double),
                ("r_in_au", C.c_double), ("r_out_au", C.c_double), ("energy_law", C.c_int32),
                ("mu_law", C.c_int32), ("scatter_law", C.c_int32), ("pad0", C.c_int32)]


class TallyDesc(C.Structure):
    _fields_ = [("cadence", C.c_int32), ("n_mu", C.c_int32), ("n_E", C.c_int32), ("n_r", C.c_int32),
                ("n_age", C.c_int32), ("pad0", C.c_int32), ("t_start_s", C.c_double),
                ("E_lo_keV", C.c_double), ("E_hi_keV", C.c_double), ("r_lo_au", C.c_double),
                ("r_hi_au", C.c_double), ("age_max_s", C.c_double), ("rwin_lo_au", C.c_double),
                ("rwin_hi_au", C.c_double), ("age_young_s", C.c_double)]


_U32P = C.POINTER(C.c_uint32)
_U64P = C.POINTER(C.c_uint64)
_DP = C.POINTER(C.c_double)


class TallyOut(C.Structure):
    _fields_ = [("h_mer", _U32P), ("h_age", _U32P), ("h_pad", _U32P), ("m_cnt", _U64P),
                ("m_sin2", _U64P), ("n_seen", _U64P)]


class ParticleSoA(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, _DP) for k in (
        "x", "y", "z", "u", "mub", "F0", "F1", "vpar", "s_rem", "h_prev", "t_birth", "u_inj",
        "mub_inj")] + [(k, _U32P) for k in ("id", "ens", "event", "ncoll", "flags")]


class StatsOut(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("step", C.c_int64), ("t", C.c_double),
                ("particle_steps", C.c_uint64), ("collisions", C.c_uint64),
                ("rebirths", C.c_uint64), ("flags_or", C.c_uint32), ("pad0", C.c_uint32),
                ("kernel_launches", C.c_uint64), ("push_launches", C.c_uint64),
                ("push_ms", C.c_double), ("sorts", C.c_uint64), ("sort_ms", C.c_double),
                ("field_evals", C.c_uint64), ("field_ms", C.c_double)]


class SirenDesc(C.Structure):
    _fields_ = [("omega0", C.c_double), ("r_max_au", C.c_double), ("B_scale", C.c_double),
                ("E_scale", C.c_double)]


class FitDesc(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("samples_on_device", C.c_int32), ("pad", C.c_int32),
                ("batch", C.c_int64), ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


SIREN_NPARAMS = 200456
FIELD_GRID, FIELD_SIREN, FIELD_GRID_SAMPLED = 0, 1, 2


class LaunchChoice(C.Structure):
    _fields_ = [("block", C.c_int32), ("grid_waves", C.c_int32), ("steps_per_launch", C.c_int32),
                ("sort_every", C.c_int32), ("particle_steps_per_s", C.c_double),
                ("trials", C.c_int32), ("pad0", C.c_int32)]


EXPORTS = ("gc_create", "gc_destroy", "gc_last_error", "gc_field_load", "gc_particles_inject",
           "gc_advance", "gc_tally", "gc_particles_get", "gc_particles_set", "gc_stats",
           "gc_set_launch", "gc_sort", "gc_version", "gc_set_clock", "gc_advance_noalloc",
           "gc_set_graph", "gc_autotune", "gc_gemm_bf16_tn", "gc_gemm_bf16", "gc_siren_set", "gc_siren_get",
           "gc_siren_eval", "gc_siren_field", "gc_field_targets", "gc_siren_loss_grad", "gc_field_fit",
           "gc_field_select", "gc_field_load_next", "gc_fma_peak")

_lib = None


def load(path: str | None = None):
    """Load libgcpush.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgcpush.so not found at {path}: run __graft_entry__.build() or "
                           "paper_2403_06706_gb300.gcpush.build() first")
    L = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "gc_create": (C.c_int, [C.POINTER(vp), C.POINTER(Options)]),
        "gc_destroy": (None, [vp]),
        "gc_last_error": (C.c_char_p, []),
        "gc_field_load": (C.c_int, [vp, C.POINTER(GridDesc), vp, C.c_int]),
        "gc_field_load_next": (C.c_int, [vp, vp, C.c_int, C.c_double, C.c_double]),
        "gc_particles_inject": (C.c_int, [vp, C.POINTER(EnsembleDesc), C.c_int]),
        "gc_advance": (C.c_int, [vp, C.c_double, C.c_int64, C.c_double]),
        "gc_tally": (C.c_int, [vp, C.POINTER(TallyDesc), C.POINTER(TallyOut)]),
        "gc_particles_get": (C.c_int, [vp, C.POINTER(ParticleSoA)]),
        "gc_particles_set": (C.c_int, [vp, C.POINTER(ParticleSoA)]),
        "gc_stats": (C.c_int, [vp, C.POINTER(StatsOut)]),
        "gc_set_launch": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "gc_set_graph": (C.c_int, [vp, C.c_int]),
        "gc_gemm_bf16_tn": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]),
        "gc_gemm_bf16": (C.c_int, [vp, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   vp]),
        "gc_autotune": (C.c_int, [vp, C.c_double, C.c_int64, C.POINTER(LaunchChoice)]),
        "gc_siren_set": (C.c_int, [vp, C.POINTER(SirenDesc), vp, C.c_int]),
        "gc_siren_get": (C.c_int, [vp, vp]),
        "gc_siren_eval": (C.c_int, [vp, vp, C.c_int64, vp, vp]),
        "gc_siren_field": (C.c_int, [vp, vp, C.c_int64, vp]),
        "gc_field_targets": (C.c_int, [vp, vp, C.c_int64, vp]),
        "gc_siren_loss_grad": (C.c_int, [vp, vp, vp, C.c_int64, vp, C.POINTER(C.c_double)]),
        "gc_field_fit": (C.c_int, [vp, C.POINTER(FitDesc), C.c_int64, C.c_int, vp]),
        "gc_field_select": (C.c_int, [vp, C.c_int]),
        "gc_sort": (C.c_int, [vp]),
        "gc_version": (C.c_int, []),
        "gc_set_clock": (C.c_int, [vp, C.c_double, C.c_int64]),
        "gc_fma_peak": (C.c_int, [C.c_int, _DP, _DP]),
        "gc_advance_noalloc": (C.c_int, [C.POINTER(Options), C.POINTER(GridDesc), vp,
                                         C.POINTER(EnsembleDesc), C.c_int, C.POINTER(ParticleSoA),
                                         C.c_double, C.c_int64, C.c_double, C.c_int64, C.c_double,
                                         C.POINTER(StatsOut)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def fma_peak(device: int = 0) -> tuple[float, float]:
    """Measured FP32 and FP64 FMA throughput of the device (TFLOP/s), gc_fma_peak."""
    a, b = C.c_double(), C.c_double()
    _check(load().gc_fma_peak(int(device), C.byref(a), C.byref(b)), "gc_fma_peak")
    return a.value, b.value


class GcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {GC_ERR.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int, where: str):
    if rc != GC_OK:
        raise GcError(rc, where, load().gc_last_error().decode(errors="replace"))


def ensemble_desc(e: EnsembleSpec) -> EnsembleDesc:
    d = EnsembleDesc()
    d.count = e.count
    d.r0_au, d.lat_deg, d.lon_deg = e.r0_au, e.lat_deg, e.lon_deg
    d.E0_keV, d.E_lo_keV, d.E_hi_keV, d.E_index = e.E0_keV, e.E_lo_keV, e.E_hi_keV, e.E_index
    d.lambda_au = e.lam_au
    d.r_in_au = e.r_in
    d.r_out_au = e.r_out_au
    d.energy_law, d.mu_law, d.scatter_law = e.energy_law, e.mu_law, e.scatter_law
    return d


F64_STATE = ("x", "y", "z", "u", "mub", "vpar", "s_rem", "h_prev", "t_birth", "u_inj", "mub_inj")
U32_STATE = ("id", "ens", "event", "ncoll", "flags")


class Context:
    """One libgcpush context (one device, one stream)."""

    def __init__(self, precision: int = PREC_FP32_MIXED, device: int = 0, stream=None, seed: int = 0,
                 collision_form: int = 0, drift_mask: int = 0, no_scatter: bool = False,
                 no_rebirth: bool = False, dt_init: float = 0.5, charge: float = 0.0,
                 mass: float = 0.0, id_base: int = 0, wind_u: float = 0.0):
        L = load()
        o = Options()
        o.precision, o.device = precision, device
        o.stream = _stream_ptr(stream)
        o.seed = seed
        o.collision_form, o.drift_mask = collision_form, drift_mask
        o.no_scatter, o.no_rebirth = int(no_scatter), int(no_rebirth)
        o.charge, o.mass, o.dt_init = charge, mass, dt_init
        o.id_base = id_base
        o.wind_u = wind_u
        h = C.c_void_p()
        _check(L.gc_create(C.byref(h), C.byref(o)), "gc_create")
        self._h = h
        self.precision = precision
        self.n_ens = 0
        self._tally = None

    def close(self):
        if getattr(self, "_h", None):
            load().gc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # field -------------------------------------------------------------------
    def field_load(self, nodes, r_min_au: float, r_max_au: float, ideal=True):
        """nodes: [n_ph][n_th][n_r][8] float32/float64, numpy (host) or torch CUDA tensor.
        ideal: True (E_par = 0), False (E_par = E.b) or 2 (two-fluid: E_par = -b.grad(Phi))."""
        g = GridDesc()
        on_dev = 0
        if hasattr(nodes, "is_cuda"):  # torch tensor
            assert nodes.is_contiguous() and nodes.dim() == 4 and nodes.shape[3] == 8
            g.n_ph, g.n_th, g.n_r = int(nodes.shape[0]), int(nodes.shape[1]), int(nodes.shape[2])
            g.dtype = DTYPE_F64 if str(nodes.dtype) == "torch.float64" else DTYPE_F32
            ptr = C.c_void_p(nodes.data_ptr())
            on_dev = 1 if nodes.is_cuda else 0
        else:
            nodes = np.ascontiguousarray(nodes)
            assert nodes.ndim == 4 and nodes.shape[3] == 8
            assert nodes.dtype in (np.float32, np.float64)
            g.n_ph, g.n_th, g.n_r = nodes.shape[:3]
            g.dtype = DTYPE_F64 if nodes.dtype == np.float64 else DTYPE_F32
            ptr = C.c_void_p(nodes.ctypes.data)
        g.r_min_au, g.r_max_au = r_min_au, r_max_au
        g.ideal = 2 if ideal == 2 else (1 if ideal else 0)
        _check(load().gc_field_load(self._h, C.byref(g), ptr, on_dev), "gc_field_load")
        self._grid_keep = nodes
        self._grid_shape = (g.n_ph, g.n_th, g.n_r, 8, g.dtype)

    def field_load_next(self, nodes, t0_s: float, t1_s: float):
        """Second snapshot of the loaded field (same shape and dtype), the two at times t0_s and
        t1_s: the field becomes linear in time between them and holds the nearer one outside."""
        if hasattr(nodes, "is_cuda"):
            assert nodes.is_contiguous()
            dt = DTYPE_F64 if str(nodes.dtype) == "torch.float64" else DTYPE_F32
            shape = tuple(int(v) for v in nodes.shape) + (dt,)
            ptr, on_dev = C.c_void_p(nodes.data_ptr()), (1 if nodes.is_cuda else 0)
        else:
            nodes = np.ascontiguousarray(nodes)
            dt = DTYPE_F64 if nodes.dtype == np.float64 else DTYPE_F32
            shape = tuple(nodes.shape) + (dt,)
            ptr, on_dev = C.c_void_p(nodes.ctypes.data), 0
        if shape != getattr(self, "_grid_shape", None):
            raise ValueError("field_load_next: snapshot %s does not match the loaded grid %s"
                             % (shape, getattr(self, "_grid_shape", None)))
        _check(load().gc_field_load_next(self._h, ptr, on_dev, float(t0_s), float(t1_s)), "gc_field_load_next")
        self._grid_keep1 = nodes

    # particles ---------------------------------------------------------------
    def inject(self, ensembles):
        arr = (EnsembleDesc * len(ensembles))(*[ensemble_desc(e) for e in ensembles])
        _check(load().gc_particles_inject(self._h, arr, len(ensembles)), "gc_particles_inject")
        self.n_ens += len(ensembles)

    def advance(self, dt: float, n_steps: int, lambda_au: float = 0.0):
        _check(load().gc_advance(self._h, dt, int(n_steps), lambda_au), "gc_advance")

    def set_launch(self, block: int = 0, steps_per_launch: int = 0, sort_every: int = 0,
                   grid_waves: int = 1):
        _check(load().gc_set_launch(self._h, block, steps_per_launch, sort_every, grid_waves),
               "gc_set_launch")

    def set_graph(self, enable: bool = True):
        _check(load().gc_set_graph(self._h, int(enable)), "gc_set_graph")

    def autotune(self, dt: float, trial_steps: int = 200) -> dict:
        b = LaunchChoice()
        _check(load().gc_autotune(self._h, dt, int(trial_steps), C.byref(b)), "gc_autotune")
        return {k: getattr(b, k) for k, _ in LaunchChoice._fields_ if k != "pad0"}

    def sort(self):
        _check(load().gc_sort(self._h), "gc_sort")

    def set_clock(self, t: float, step: int):
        _check(load().gc_set_clock(self._h, float(t), int(step)), "gc_set_clock")

    def stats(self) -> dict:
        s = StatsOut()
        _check(load().gc_stats(self._h, C.byref(s)), "gc_stats")
        return {k: getattr(s, k) for k, _ in StatsOut._fields_ if k != "pad0"}

    @property
    def n(self) -> int:
        return self.stats()["n_particles"]

    def get_state(self, out: dict | None = None) -> dict:
        """Particle state in ascending id order; fills ``out`` (e.g. pinned arrays) if given."""
        n = self.n
        a = out if out is not None else state_buffers(n)
        s = ParticleSoA()
        s.n = n
        for k in F64_STATE + ("F0", "F1"):
            assert a[k].dtype == np.float64 and a[k].flags.c_contiguous and a[k].shape[-1] == n
            setattr(s, k, a[k].ctypes.data_as(_DP))
        for k in U32_STATE:
            assert a[k].dtype == np.uint32 and a[k].flags.c_contiguous and a[k].shape[-1] == n
            setattr(s, k, a[k].ctypes.data_as(_U32P))
        _check(load().gc_particles_get(self._h, C.byref(s)), "gc_particles_get")
        return a

    def set_state(self, a: dict):
        n = a["x"].shape[0]
        s = ParticleSoA()
        s.n = n
        keep = {}
        for k in F64_STATE + ("F0", "F1"):
            keep[k] = np.ascontiguousarray(a[k], dtype=np.float64)
            setattr(s, k, keep[k].ctypes.data_as(_DP))
        for k in U32_STATE:
            keep[k] = np.ascontiguousarray(a[k], dtype=np.uint32)
            setattr(s, k, keep[k].ctypes.data_as(_U32P))
        _check(load().gc_particles_set(self._h, C.byref(s)), "gc_particles_set")

    # tallies -----------------------------------------------------------------
    # neural field --------------------------------------------------------------
    def siren_set(self, params, omega0: float = 30.0, r_max_au: float = 2.5, B_scale: float = 1.0,
                  E_scale: float = 1.0):
        """Load SIREN parameters (numpy float32 array or torch CUDA tensor of SIREN_NPARAMS)."""
        d = SirenDesc(omega0, r_max_au, B_scale, E_scale)
        if hasattr(params, "data_ptr"):
            assert params.numel() == SIREN_NPARAMS and params.is_contiguous()
            _check(load().gc_siren_set(self._h, C.byref(d), params.data_ptr(), 1), "gc_siren_set")
        else:
            a = np.ascontiguousarray(params, dtype=np.float32)
            assert a.size == SIREN_NPARAMS
            _check(load().gc_siren_set(self._h, C.byref(d), a.ctypes.data, 0), "gc_siren_set")

    def siren_get(self) -> np.ndarray:
        a = np.empty(SIREN_NPARAMS, dtype=np.float32)
        _check(load().gc_siren_get(self._h, a.ctypes.data), "gc_siren_get")
        return a

    def siren_eval(self, x, y, J=None):
        """Raw outputs at x (torch CUDA float32 n x 3) into y (n x 8) and J (n x 8 x 3)."""
        _check(load().gc_siren_eval(self._h, x.data_ptr(), x.shape[0], y.data_ptr(),
                                    None if J is None else J.data_ptr()), "gc_siren_eval")

    def siren_field(self, x, field):
        _check(load().gc_siren_field(self._h, x.data_ptr(), x.shape[0], field.data_ptr()), "gc_siren_field")

    def field_targets(self, x, t):
        _check(load().gc_field_targets(self._h, x.data_ptr(), x.shape[0], t.data_ptr()), "gc_field_targets")

    def siren_loss_grad(self, x, t, grad=None) -> float:
        loss = C.c_double()
        _check(load().gc_siren_loss_grad(self._h, x.data_ptr(), t.data_ptr(), x.shape[0],
                                         None if grad is None else grad.data_ptr(), C.byref(loss)),
               "gc_siren_loss_grad")
        return loss.value

    def field_fit(self, samples, n_epochs: int, batch: int = 65536, lr: float = 1e-4, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8) -> np.ndarray:
        """Fit the network to the loaded grid at samples (n x 3 scaled positions; numpy or
        torch CUDA); returns the per-epoch mean loss."""
        on_dev = hasattr(samples, "data_ptr")
        if on_dev:
            ptr, n = samples.data_ptr(), samples.shape[0]
        else:
            samples = np.ascontiguousarray(samples, dtype=np.float32)
            ptr, n = samples.ctypes.data, samples.shape[0]
        f = FitDesc(ptr, int(on_dev), 0, batch, lr, beta1, beta2, eps)
        out = np.zeros(max(n_epochs, 1), dtype=np.float32)
        _check(load().gc_field_fit(self._h, C.byref(f), n, n_epochs, out.ctypes.data), "gc_field_fit")
        return out[:n_epochs]

    def field_select(self, source: int):
        _check(load().gc_field_select(self._h, source), "gc_field_select")

    def tally_arm(self, cadence=100, n_mu=32, n_E=32, n_r=64, n_age=32, t_start_s=0.0,
                  E_lo_keV=5.0, E_hi_keV=600.0, r_lo_au=0.1, r_hi_au=2.5, age_max_s=86400.0,
                  rwin_lo_au=0.9, rwin_hi_au=1.1, age_young_s=1200.0):
        t = TallyDesc()
        t.cadence, t.n_mu, t.n_E, t.n_r, t.n_age = cadence, n_mu, n_E, n_r, n_age
        t.t_start_s, t.E_lo_keV, t.E_hi_keV = t_start_s, E_lo_keV, E_hi_keV
        t.r_lo_au, t.r_hi_au, t.age_max_s = r_lo_au, r_hi_au, age_max_s
        t.rwin_lo_au, t.rwin_hi_au, t.age_young_s = rwin_lo_au, rwin_hi_au, age_young_s
        _check(load().gc_tally(self._h, C.byref(t), None), "gc_tally")
        self._tally = (t, max(1, self.n_ens))

    def tally_read(self) -> dict:
        t, ne = self._tally
        out = {
            "h_mer": np.zeros((ne, t.n_mu, t.n_E, t.n_r), dtype=np.uint32),
            "h_age": np.zeros((ne, t.n_age, t.n_E), dtype=np.uint32),
            "h_pad": np.zeros((ne, t.n_mu), dtype=np.uint32),
            "m_cnt": np.zeros((ne, t.n_r), dtype=np.uint64),
            "m_sin2": np.zeros((ne, t.n_r), dtype=np.uint64),
            "n_seen": np.zeros(2, dtype=np.uint64),
        }
        o = TallyOut()
        for k in ("h_mer", "h_age", "h_pad"):
            setattr(o, k, out[k].ctypes.data_as(_U32P))
        for k in ("m_cnt", "m_sin2", "n_seen"):
            setattr(o, k, out[k].ctypes.data_as(_U64P))
        _check(load().gc_tally(self._h, None, C.byref(o)), "gc_tally")
        return out


def state_buffers(n: int, alloc=np.zeros) -> dict:
    """Host arrays for one particle state (``alloc(shape, dtype)``, e.g. a pinned allocator)."""
    a = {k: alloc((n,), np.float64) for k in F64_STATE}
    a.update({k: alloc((n,), np.uint32) for k in U32_STATE})
    a["F0"] = alloc((4, n), np.float64)
    a["F1"] = alloc((4, n), np.float64)
    return a


def state_nbytes(a: dict) -> int:
    return int(sum(v.nbytes for v in a.values()))


def gemm_bf16_tn(A, B, C, split_k: int = 1, accumulate: bool = False, stream=None):
    """C = A B^T (or C += A B^T) on the tensor cores; torch CUDA tensors (A, B bf16)."""
    M, K = A.shape
    N = B.shape[0]
    assert B.shape[1] == K and C.shape == (M, N) and A.is_contiguous() and B.is_contiguous()
    _check(load().gc_gemm_bf16_tn(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, split_k,
                                  int(accumulate), _stream_ptr(stream)), "gc_gemm_bf16_tn")


def gemm_bf16(A, B, C, a_mn: bool = False, b_mn: bool = False, split_k: int = 1, accumulate: bool = False,
              stream=None):
    """C = op(A) op(B)^T on the tensor cores: op(A) is A (M x K) or, with a_mn, A^T for A
    given as K x M; op(B) likewise N x K or K x N. torch CUDA tensors (A, B bf16, C fp32)."""
    M, K = (A.shape[1], A.shape[0]) if a_mn else A.shape
    N, Kb = (B.shape[1], B.shape[0]) if b_mn else B.shape
    assert Kb == K and C.shape == (M, N) and A.is_contiguous() and B.is_contiguous()
    _check(load().gc_gemm_bf16(A.data_ptr(), int(a_mn), B.data_ptr(), int(b_mn), C.data_ptr(), M, N, K, split_k,
                               int(accumulate), _stream_ptr(stream)), "gc_gemm_bf16")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream

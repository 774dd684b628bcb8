"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  If the compiled library is missing or no GPU is usable, the
calls raise; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FP64, FP32, FP16S = 0, 1, 2
STEP_DIRECT = 1
OK, ERR_BADPARAM, ERR_OOM, ERR_DIVERGED, ERR_CUDA, ERR_STATE = 0, -1, -2, -3, -4, -5
WARN_NOT_CONVERGED = 1

FIELD_IDS = {
    "f": 0, "h": 1, "g": 2, "l": 3, "fs_prev": 4, "mdot_prev": 5, "Q_prev": 6,
    "psiux": 7, "psiuy": 8, "p": 9, "S": 10, "psi": 11, "fsolid": 12, "T": 13,
    "phi": 14, "H": 15, "sigma": 16,
}
FIELD_PLANES = {"f": 9, "h": 9, "g": 9, "l": 5}

# Every entry point the header declares (checked by the CPU test suite).
EXPORTS = [
    "lbm_last_error", "lbm_create", "lbm_init_droplet", "lbm_init_psi", "lbm_step",
    "lbm_observables", "lbm_observables_async", "lbm_observables_fetch", "lbm_get_field",
    "lbm_set_field", "lbm_state_bytes", "lbm_export_state", "lbm_import_state",
    "lbm_step_count", "lbm_configure", "lbm_destroy", "lbm_batch_create", "lbm_batch_step",
    "lbm_batch_tile_rows", "lbm_batch_destroy", "lbm_observables_noalloc",
    "lbm_substrate_heat_flux", "lbm_observables_to_host", "lbm_sync", "lbm_observables_deferred",
    "lbm_presolve", "lbm_device_bytes", "lbm_round_half_sr",
]


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("k_e", C.c_int32), ("precision", C.c_int32),
        ("W", C.c_double), ("M", C.c_double), ("gamma", C.c_double),
        ("rho_l", C.c_double), ("rho_lg", C.c_double), ("rho_sl", C.c_double),
        ("mu_l", C.c_double), ("mu_lg", C.c_double),
        ("Ste", C.c_double), ("alpha_l", C.c_double), ("alpha_lg", C.c_double),
        ("cp_l", C.c_double), ("cp_s", C.c_double), ("cp_g", C.c_double),
        ("T_m", C.c_double), ("T_w", C.c_double), ("T_init", C.c_double),
        ("CaE", C.c_double), ("R_sigma", C.c_double), ("S_eps", C.c_double),
        ("eps_g", C.c_double), ("sigma_g", C.c_double), ("R0", C.c_double),
        ("theta_deg", C.c_double), ("alpha_sl", C.c_double),
    ]


class Obs(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("Fo", C.c_double), ("mass", C.c_double),
        ("enthalpy", C.c_double), ("charge", C.c_double), ("solid", C.c_double),
        ("frozen_fraction", C.c_double), ("height", C.c_double), ("width", C.c_double),
        ("aspect", C.c_double), ("R_tr", C.c_double), ("front", C.c_double),
        ("t_fre", C.c_int64), ("Fo_fre", C.c_double), ("status", C.c_int32),
        ("reserved", C.c_int32), ("Pe", C.c_double), ("Qdot", C.c_double),
    ]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it first if allowed and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"GPU library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    P = C.POINTER
    vp = C.c_void_p
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_create.argtypes = [P(Params), vp, P(vp)]
    L.lbm_init_droplet.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_int32]
    L.lbm_init_psi.argtypes = [vp, P(C.c_double), C.c_int32]
    L.lbm_step.argtypes = [vp, C.c_int64]
    L.lbm_observables.argtypes = [vp, P(Obs)]
    L.lbm_observables_async.argtypes = [vp]
    L.lbm_observables_fetch.argtypes = [vp, P(Obs)]
    L.lbm_observables_to_host.argtypes = [vp, vp]
    L.lbm_sync.argtypes = [vp]
    L.lbm_observables_deferred.argtypes = [vp, vp]
    L.lbm_presolve.argtypes = [vp, C.c_double, C.c_int32, P(C.c_int32), P(C.c_double)]
    L.lbm_get_field.argtypes = [vp, C.c_int32, P(C.c_double)]
    L.lbm_set_field.argtypes = [vp, C.c_int32, P(C.c_double)]
    L.lbm_state_bytes.restype = C.c_size_t
    L.lbm_state_bytes.argtypes = [vp]
    L.lbm_export_state.argtypes = [vp, vp, C.c_size_t]
    L.lbm_import_state.argtypes = [vp, vp, C.c_size_t]
    L.lbm_configure.argtypes = [vp, C.c_int32, C.c_int32]
    L.lbm_step_count.restype = C.c_int64
    L.lbm_step_count.argtypes = [vp]
    L.lbm_device_bytes.restype = C.c_size_t
    L.lbm_device_bytes.argtypes = [vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_batch_create.argtypes = [P(vp), C.c_int32, vp, C.c_int32, P(vp)]
    L.lbm_batch_step.argtypes = [vp, C.c_int64]
    L.lbm_batch_tile_rows.restype = C.c_int32
    L.lbm_batch_tile_rows.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_substrate_heat_flux.argtypes = [vp, P(C.c_double)]
    L.lbm_round_half_sr.argtypes = [vp, vp, vp, C.c_int64, vp]
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise LBMError(rc, load().lbm_last_error().decode(errors="replace"))
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: dict) -> Params:
    out = Params()
    names = {n for n, _ in Params._fields_}
    for k, v in p.items():
        if k in names:
            setattr(out, k, v)
    return out


def _stream_handle(stream):
    """A cudaStream_t as an integer: None -> torch's current stream (if torch
    is importable with CUDA), else the legacy default stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def round_half_sr(v, r, stream=None):
    """The half-storage stochastic rounding of the float32 device tensor v
    with the random bits r (int32 device tensor of the same length; its low
    13 bits are used): the 16 bits of each half, as an int16 device tensor.
    Enqueued on `stream` (default: torch's current stream)."""
    import torch
    if v.dtype != torch.float32 or r.dtype != torch.int32 or not v.is_cuda or not r.is_cuda:
        raise ValueError("v must be a float32 and r an int32 CUDA tensor")
    if v.numel() != r.numel() or not v.is_contiguous() or not r.is_contiguous():
        raise ValueError("v and r must be contiguous and of the same length")
    out = torch.empty(v.numel(), dtype=torch.int16, device=v.device)
    L = load()
    _check(L.lbm_round_half_sr(C.c_void_p(v.data_ptr()), C.c_void_p(r.data_ptr()), C.c_void_p(out.data_ptr()),
                               v.numel(), C.c_void_p(_stream_handle(stream))))
    return out


class Simulation:
    """One lattice instance on the GPU (``lbm_create`` ... ``lbm_destroy``)."""

    def __init__(self, params: dict, stream=None):
        L = load()
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._p = make_params(params)
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        _check(L.lbm_create(C.byref(self._p), C.c_void_p(self.stream), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, variant=STEP_DIRECT, tile_rows=4):
        _check(load().lbm_configure(self._h, int(variant), int(tile_rows)))

    def init_droplet(self, R, xc, yc, presolve=0):
        _check(load().lbm_init_droplet(self._h, float(R), float(xc), float(yc), int(presolve)))

    def init_psi(self, psi, presolve=0):
        a = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.ny, self.nx)
        _check(load().lbm_init_psi(self._h, _dp(a), int(presolve)))

    def step(self, n=1):
        _check(load().lbm_step(self._h, int(n)))

    @property
    def t(self):
        return int(load().lbm_step_count(self._h))

    def observables(self) -> dict:
        o = Obs()
        rc = load().lbm_observables(self._h, C.byref(o))
        if rc not in (OK, ERR_DIVERGED):
            _check(rc)
        return o.as_dict()

    def substrate_heat_flux(self) -> np.ndarray:
        """Local heat flux through the cold substrate, one value per column
        (Sec. 4.3)."""
        out = np.zeros(self.nx)
        _check(load().lbm_substrate_heat_flux(self._h, _dp(out)))
        return out

    def observables_async(self):
        _check(load().lbm_observables_async(self._h))

    def observables_fetch(self) -> dict:
        o = Obs()
        rc = load().lbm_observables_fetch(self._h, C.byref(o))
        if rc not in (OK, ERR_DIVERGED):
            _check(rc)
        return o.as_dict()

    def observables_to_host(self, addr: int):
        """Enqueue the observables and their copy to the host address `addr`
        (an lbm_obs, page-locked for an asynchronous copy); read it with
        `Obs.from_address(addr)` after `sync()`."""
        _check(load().lbm_observables_to_host(self._h, C.c_void_p(addr)))

    def presolve(self, tol: float, max_sweeps: int) -> dict:
        """Potential sweeps until phi changes by less than tol (relative to
        the electrode difference) over one sweep; see lbm_presolve."""
        n, r = C.c_int32(0), C.c_double(0.0)
        rc = load().lbm_presolve(self._h, float(tol), int(max_sweeps), C.byref(n), C.byref(r))
        if rc < 0:
            _check(rc)
        return {"converged": rc == OK, "sweeps": int(n.value), "residual": float(r.value)}

    def observables_deferred(self, addr: int = 0):
        """Request the observables of the current state, reduced inside the
        next step's kernel; fetch with `observables_fetch()`, or pass a host
        address (an lbm_obs) to receive them there after `sync()`."""
        _check(load().lbm_observables_deferred(self._h, C.c_void_p(addr) if addr else None))

    def sync(self):
        _check(load().lbm_sync(self._h))

    def get(self, name: str) -> np.ndarray:
        planes = FIELD_PLANES.get(name, 1)
        out = np.empty((planes, self.ny, self.nx), dtype=np.float64)
        _check(load().lbm_get_field(self._h, FIELD_IDS[name], _dp(out)))
        return out if planes > 1 else out[0]

    def set(self, name: str, values):
        planes = FIELD_PLANES.get(name, 1)
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(planes, self.ny, self.nx)
        _check(load().lbm_set_field(self._h, FIELD_IDS[name], _dp(a)))

    def state_bytes(self) -> int:
        return int(load().lbm_state_bytes(self._h))

    def device_bytes(self) -> int:
        """Device memory the instance holds (lbm_device_bytes)."""
        return int(load().lbm_device_bytes(self._h))

    def export_state(self, buf=None) -> np.ndarray:
        n = self.state_bytes()
        if buf is None:
            buf = np.empty(n, dtype=np.uint8)
        _check(load().lbm_export_state(self._h, C.c_void_p(buf.ctypes.data), n))
        return buf

    def import_state(self, buf):
        """`buf`: numpy uint8 array or a host pointer (int) with state_bytes() bytes."""
        n = self.state_bytes()
        ptr = buf if isinstance(buf, int) else buf.ctypes.data
        _check(load().lbm_import_state(self._h, C.c_void_p(ptr), n))


class Batch:
    """Many instances stepped by one launch per step (``lbm_batch_*``)."""

    def __init__(self, sims, stream=None, tile_rows=0):
        L = load()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.handle.value for s in self.sims])
        b = C.c_void_p()
        st = _stream_handle(stream) if stream is not None else self.sims[0].stream
        _check(L.lbm_batch_create(arr, len(self.sims), C.c_void_p(st), int(tile_rows), C.byref(b)))
        self._b = b

    @property
    def tile_rows(self):
        return int(load().lbm_batch_tile_rows(self._b))

    def step(self, n=1):
        _check(load().lbm_batch_step(self._b, int(n)))

    def close(self):
        if getattr(self, "_b", None):
            load().lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Plain FP64 CPU oracle for the phase-field LB electrofreezing step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never calls it and shares no code with it: the C
source in ``lbm_oracle.c`` is a separate, slow, loop-by-loop transcription of
the paper's equations (Secs. 2-3, Algorithm 1) in double precision.

Every function is pinned by a closed form, an invariant or a value the
paper prints (tests/test_oracle_pins.py); tests/test_oracle_mutants.py
checks that those pins reject copies with a term dropped or flipped.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")

# field ids (same numbering as the library's public header)
FIELD_IDS = {
    "f": 0, "h": 1, "g": 2, "l": 3, "fs_prev": 4, "mdot_prev": 5, "Q_prev": 6,
    "psiux": 7, "psiuy": 8, "p": 9, "S": 10, "psi": 11, "fsolid": 12, "T": 13,
    "phi": 14, "H": 15, "sigma": 16,
}
FIELD_PLANES = {"f": 9, "h": 9, "g": 9, "l": 5}


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("k_e", C.c_int32), ("reserved", C.c_int32),
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


class OrcDerived(C.Structure):
    _fields_ = [
        ("rho", C.c_double * 3), ("mu", C.c_double * 3), ("kth", C.c_double * 3),
        ("cp", C.c_double * 3), ("eps", C.c_double * 3), ("sig", C.c_double * 3),
        ("L", C.c_double), ("Cref", C.c_double), ("kappa", C.c_double), ("beta", C.c_double),
        ("tau_f", C.c_double), ("E0", C.c_double), ("phi_bot", C.c_double),
        ("phi_top", C.c_double), ("wet", C.c_double), ("alpha_s", C.c_double),
    ]


class OrcObs(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("Fo", C.c_double), ("mass", C.c_double),
        ("enthalpy", C.c_double), ("charge", C.c_double), ("solid", C.c_double),
        ("frozen_fraction", C.c_double), ("height", C.c_double), ("width", C.c_double),
        ("aspect", C.c_double), ("R_tr", C.c_double), ("front", C.c_double),
        ("t_fre", C.c_int64), ("Fo_fre", C.c_double), ("status", C.c_int32),
        ("reserved", C.c_int32), ("Pe", C.c_double), ("Qdot", C.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, plain -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def build_variant(source: str, out_dir: str, tag: str):
    """Compile another oracle source text (a copy with one change, for the
    mutation tests of the pins) the way build() compiles the oracle, and
    load it.  Returns the library to pass as Oracle(..., lib=...)."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, f"lbm_oracle_{tag}.c")
    with open(src, "w") as fh:
        fh.write(source)
    so = os.path.join(out_dir, f"liblbm_oracle_{tag}.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", so,
                    src, "-lm"], check=True)
    return _load(so)


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _load(path):
    L = C.CDLL(path)
    P = C.POINTER
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [P(OrcParams)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_derive.argtypes = [P(OrcParams), P(OrcDerived)]
    L.orc_get_derived.argtypes = [C.c_void_p, P(OrcDerived)]
    L.orc_step.argtypes = [C.c_void_p, C.c_int64]
    L.orc_get_step.restype = C.c_int64
    L.orc_get_step.argtypes = [C.c_void_p]
    L.orc_init_droplet.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int32]
    L.orc_init_psi.argtypes = [C.c_void_p, P(C.c_double), C.c_int32]
    L.orc_get_field.argtypes = [C.c_void_p, C.c_int32, P(C.c_double)]
    L.orc_set_field.argtypes = [C.c_void_p, C.c_int32, P(C.c_double)]
    L.orc_observables.argtypes = [C.c_void_p, P(OrcObs)]
    L.orc_heat_flux.argtypes = [C.c_void_p, P(C.c_double)]
    L.orc_lattice.argtypes = [P(C.c_int32), P(C.c_int32), P(C.c_double)]
    L.orc_enthalpy_inversion.argtypes = [C.c_double] * 5 + [P(C.c_double), P(C.c_double)]
    L.orc_stencils.argtypes = [C.c_int32, C.c_int32, P(C.c_double), C.c_int32, C.c_double,
                               C.c_double, C.c_double, P(C.c_double), P(C.c_double),
                               P(C.c_double)]
    L.orc_pointwise.argtypes = [C.c_double] * 23 + [P(C.c_double)] * 6
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: dict) -> OrcParams:
    out = OrcParams()
    names = {n for n, _ in OrcParams._fields_}
    for k, v in p.items():
        if k in names:
            setattr(out, k, v)
    return out


def derive(p: dict) -> dict:
    """Lattice-unit constants the oracle derives from a parameter dict."""
    d = OrcDerived()
    rc = lib().orc_derive(C.byref(make_params(p)), C.byref(d))
    if rc != 0:
        raise ValueError("oracle: invalid parameters")
    out = {}
    for name, _ in OrcDerived._fields_:
        v = getattr(d, name)
        out[name] = list(v) if not isinstance(v, float) else v
    return out


class Oracle:
    """One simulation instance on the CPU (FP64)."""

    def __init__(self, params: dict, lib=None):
        self.params = dict(params)
        self._p = make_params(params)
        self._L = lib if lib is not None else globals()["lib"]()
        self._h = self._L.orc_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.nx, self.ny = int(params["nx"]), int(params["ny"])

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_droplet(self, R, xc, yc, presolve=0):
        self._L.orc_init_droplet(self._h, float(R), float(xc), float(yc), int(presolve))

    def init_psi(self, psi, presolve=0):
        a = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.ny, self.nx)
        self._L.orc_init_psi(self._h, _dp(a), int(presolve))

    def step(self, n=1):
        self._L.orc_step(self._h, int(n))

    @property
    def t(self):
        return int(self._L.orc_get_step(self._h))

    def get(self, name: str) -> np.ndarray:
        planes = FIELD_PLANES.get(name, 1)
        out = np.empty((planes, self.ny, self.nx), dtype=np.float64)
        rc = self._L.orc_get_field(self._h, FIELD_IDS[name], _dp(out))
        if rc != 0:
            raise KeyError(name)
        return out if planes > 1 else out[0]

    def set(self, name: str, values: np.ndarray):
        planes = FIELD_PLANES.get(name, 1)
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(planes, self.ny, self.nx)
        rc = self._L.orc_set_field(self._h, FIELD_IDS[name], _dp(a))
        if rc != 0:
            raise KeyError(name)

    def derived(self) -> dict:
        d = OrcDerived()
        self._L.orc_get_derived(self._h, C.byref(d))
        return {n: (list(getattr(d, n)) if not isinstance(getattr(d, n), float) else getattr(d, n))
                for n, _ in OrcDerived._fields_}

    def observables(self) -> dict:
        o = OrcObs()
        self._L.orc_observables(self._h, C.byref(o))
        return o.as_dict()

    def heat_flux(self) -> np.ndarray:
        """Local substrate heat flux per column (Sec. 4.3, reading R24)."""
        out = np.zeros(self.nx)
        if self._L.orc_heat_flux(self._h, _dp(out)) != 0:
            raise ValueError("oracle: heat flux needs ny >= 3")
        return out


def lattice():
    cx = (C.c_int32 * 9)()
    cy = (C.c_int32 * 9)()
    w = (C.c_double * 9)()
    lib().orc_lattice(cx, cy, w)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:])


def enthalpy_inversion(H, psi, cp, Tm, L):
    fl = C.c_double()
    T = C.c_double()
    lib().orc_enthalpy_inversion(H, psi, cp, Tm, L, C.byref(fl), C.byref(T))
    return fl.value, T.value


def stencils(z: np.ndarray, kind=0, wet=0.0, phi_bot=0.0, phi_top=0.0):
    z = np.ascontiguousarray(z, dtype=np.float64)
    ny, nx = z.shape
    gx = np.empty_like(z)
    gy = np.empty_like(z)
    lp = np.empty_like(z)
    lib().orc_stencils(nx, ny, _dp(z), kind, wet, phi_bot, phi_top, _dp(gx), _dp(gy), _dp(lp))
    return gx, gy, lp


def pointwise(**kw):
    """All equilibria and forcing terms at one point (moment-identity tests)."""
    names = ["psi", "ux", "uy", "p", "rho", "H", "T", "cp", "Cref", "phi", "S", "Fx", "Fy",
             "rfx", "rfy", "Ftx", "Fty", "dtx", "dty", "lam", "nxv", "nyv", "divu"]
    args = [float(kw.get(n, 0.0)) for n in names]
    bufs = [np.zeros(9) for _ in range(5)] + [np.zeros(5)]
    lib().orc_pointwise(*args, *[_dp(b) for b in bufs])
    keys = ["feq", "fsrc", "heq", "hsrc", "geq", "leq"]
    return dict(zip(keys, bufs))

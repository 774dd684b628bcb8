"""Seeded synthetic workloads: parameter sets, lattice sizes and request streams.

This module holds no arithmetic of the lattice Boltzmann method.  It only
states problem set-ups (the dimensionless parameters of Sec. 5 and the
lattice choices made for them) and draws seeded random instances.  Both the
GPU library's callers and the CPU oracle's tests take their inputs from here.

Parameter dictionaries use the field names of ``lbm_params`` in
``include/lbm.h``.  Lattice choices the paper does not fix (W, M, gamma,
densities, alpha_l, ...) follow one documented reading: density and
viscosity ratio 10 (equal kinematic viscosity 0.1 in both fluids, so
tau_h = 0.8), W = 4, M = 0.1 (tau_f = 0.8), gamma = 0.01, C_p = 1 in all
phases, T_m = 0, T_w = -1 (so L = 1/Ste), alpha_l = 0.032 and
alpha_l/alpha_g = 0.2 (Sec. 5.1, Figs. 7-8), sigma_g = 1/6 (tau_l = 1 in the
gas).
"""
from __future__ import annotations

import math
import numpy as np

FP64, FP32, FP16S = 0, 1, 2
PRECISIONS = {"f64": FP64, "f32": FP32, "f16s": FP16S}

BASE = dict(
    nx=128, ny=64, k_e=1, precision=FP64,
    W=4.0, M=0.1, gamma=0.01,
    rho_l=1.0, rho_lg=10.0, rho_sl=0.9,
    mu_l=0.1, mu_lg=10.0,
    Ste=0.5, alpha_l=0.032, alpha_lg=0.2,
    cp_l=1.0, cp_s=1.0, cp_g=1.0,
    T_m=0.0, T_w=-1.0, T_init=0.0,
    CaE=0.2, R_sigma=5.0, S_eps=2.0, eps_g=1.0, sigma_g=1.0 / 6.0,
    R0=20.0, theta_deg=90.0, alpha_sl=1.0,
)

# The three electric regimes of Sec. 5 (Fig. 6): (R, S) = (sigma ratio, eps ratio)
REGIMES = {
    "OB-": (2.0, 5.0),
    "PR+": (2.0, 0.5),
    "PR-": (5.0, 9.5),
}


def params(**over) -> dict:
    p = dict(BASE)
    p.update(over)
    return p


def sessile_center(nx: int, R: float, theta_deg: float):
    """Centre of a circular cap of radius R meeting the wall y = -1/2 at
    contact angle theta (measured through the liquid), centred in x."""
    return nx / 2.0, -0.5 - R * math.cos(math.radians(theta_deg))


def droplet_psi(nx: int, ny: int, R: float, xc: float, yc: float, W: float) -> np.ndarray:
    """Initial order parameter of a circular droplet (Sec. 2): a tanh profile
    of width W around the circle of radius R centred at (xc, yc), cell (x, y)
    at (x, y).  Host copy for callers that want identical inputs on several
    back ends (lbm_init_psi)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / W)


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------

def plain_fp64_small() -> dict:
    """128x64, R = 20, theta = 90, CaE = 0.2, S = 2, R_sigma = 5, Ste = 0.5,
    2000 steps, FP64: the case the oracle finishes in seconds."""
    p = params(nx=128, ny=64, R0=20.0, theta_deg=90.0, precision=FP64)
    return dict(params=p, R=20.0, steps=2000, presolve=0)


def production(precision=FP32, regime=None, CaE=0.2) -> dict:
    """512x256, R = 80, same physics, run to freezing (about 2e5 steps)."""
    over = dict(nx=512, ny=256, R0=80.0, theta_deg=90.0, precision=precision, CaE=CaE)
    if regime is not None:
        over["R_sigma"], over["S_eps"] = REGIMES[regime]
    p = params(**over)
    return dict(params=p, R=80.0, steps=200000, presolve=0)


def precision_case(precision=FP32) -> dict:
    """1024x512, R = 160, theta = 60, field on (PR+)."""
    Rs, Se = REGIMES["PR+"]
    p = params(nx=1024, ny=512, R0=160.0, theta_deg=60.0, precision=precision,
               R_sigma=Rs, S_eps=Se)
    return dict(params=p, R=160.0, steps=0, presolve=0)


# Physical properties of Table 1 (liquid / solid), wall temperatures of Sec. 4.1.
TABLE1 = {
    "water": dict(rho=(999.0, 917.0), k=(0.581, 2.16), cp=(4220.0, 2100.0), mu=0.003,
                  sigma=0.076, L=333.4e3, T_m=0.0, T_wall=-10.0),
    "hexadecane": dict(rho=(774.0, 833.0), k=(0.15, 0.15), cp=(2310.0, 1800.0), mu=0.003,
                       sigma=0.028, L=230.0e3, T_m=18.0, T_wall=15.0),
}


def table1_dimensionless(substance: str) -> dict:
    """Dimensionless groups of a Table 1 substance: Ste = C_p,l (T_m - T_w)/L,
    rho_s/rho_l, C_p,s/C_p,l and alpha_s/alpha_l (alpha = k / (rho C_p))."""
    t = TABLE1[substance]
    (rl, rs), (kl, ks), (cl, cs) = t["rho"], t["k"], t["cp"]
    return dict(Ste=cl * (t["T_m"] - t["T_wall"]) / t["L"], rho_sl=rs / rl, cp_sl=cs / cl,
                alpha_sl=(ks / (rs * cs)) / (kl / (rl * cl)))


def table1_case(substance: str, precision=FP32, nx=512, ny=256) -> dict:
    """Sessile freezing of a Table 1 droplet without a field (Sec. 4.1): the
    liquid/solid ratios of Table 1 in lattice units (C_p,l = 1), theta = 87
    degrees, R = 0.3125 ny; gas properties and the lattice choices as in the
    base set."""
    d = table1_dimensionless(substance)
    R = 0.3125 * ny
    p = params(nx=nx, ny=ny, R0=R, theta_deg=87.0, precision=precision, CaE=0.0,
               Ste=d["Ste"], rho_sl=d["rho_sl"], cp_l=1.0, cp_s=d["cp_sl"], alpha_sl=d["alpha_sl"])
    return dict(params=p, R=R, presolve=0)


BATCH_SIZES = [(128, 64), (256, 128), (384, 192), (512, 256)]


def batched(n=64, seed=2410066570, precision=FP32) -> list:
    """n instances, sizes uniform over BATCH_SIZES, R = 0.3125 ny, CaE ~ U[0, 0.5],
    R_sigma and S_eps log-uniform on [0.2, 10], theta ~ U[60, 120], Ste ~ U[0.1, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny = BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]
        R = 0.3125 * ny
        p = params(
            nx=nx, ny=ny, R0=R, precision=precision,
            CaE=float(rng.uniform(0.0, 0.5)),
            R_sigma=float(math.exp(rng.uniform(math.log(0.2), math.log(10.0)))),
            S_eps=float(math.exp(rng.uniform(math.log(0.2), math.log(10.0)))),
            theta_deg=float(rng.uniform(60.0, 120.0)),
            Ste=float(rng.uniform(0.1, 1.0)),
        )
        out.append(dict(params=p, R=R, presolve=0))
    return out


SERVE_SIZES = [(128, 64), (256, 128), (384, 192), (512, 256), (768, 384), (1024, 512)]


def serving_stream(n=256, rate=20.0, seed=2410066571, max_ny=512, precision=FP32) -> list:
    """Poisson arrivals (mean `rate` per second) of freezing simulations with
    the batched workload's parameter draws and sizes up to 1024x512."""
    rng = np.random.default_rng(seed)
    sizes = [s for s in SERVE_SIZES if s[1] <= max_ny]
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        nx, ny = sizes[int(rng.integers(len(sizes)))]
        R = 0.3125 * ny
        p = params(
            nx=nx, ny=ny, R0=R, precision=precision,
            CaE=float(rng.uniform(0.0, 0.5)),
            R_sigma=float(math.exp(rng.uniform(math.log(0.2), math.log(10.0)))),
            S_eps=float(math.exp(rng.uniform(math.log(0.2), math.log(10.0)))),
            theta_deg=float(rng.uniform(60.0, 120.0)),
            Ste=float(rng.uniform(0.1, 1.0)),
        )
        out.append(dict(id=i, arrival=t, params=p, R=R, presolve=0))
    return out


def noise(shape, seed, scale=1.0) -> np.ndarray:
    """Seeded uniform noise on [-scale, scale] (perturbations for parity tests)."""
    rng = np.random.default_rng(seed)
    return scale * (2.0 * rng.random(shape) - 1.0)

"""Long oracle simulations behind the physics pins.

Each function runs one plain-FP64 oracle case and returns plain numbers.  They
are module-level so a ``spawn`` process pool can run them side by side; the
test session starts that pool once and shares the results.
"""
from __future__ import annotations

import math
import numpy as np


def _oracle():
    import oracle
    return oracle


def _W():
    from paper_2410_06657_gb300 import workloads
    return workloads


def layer_psi(nx, ny, h0, W):
    """Planar liquid layer of thickness h0 on the bottom wall (y = -1/2)."""
    y = np.arange(ny, dtype=np.float64)[:, None] + 0.5 + np.zeros((1, nx))
    return 0.5 + 0.5 * np.tanh(2.0 * (h0 - y) / W)


def laplace(R, W=4.0, N=64, steps=5000):
    """Static drop in the middle of an N x N box, no freezing, no field."""
    o = _oracle().Oracle(_W().params(nx=N, ny=N, T_w=0.0, CaE=0.0, R0=R, theta_deg=90.0, W=W))
    o.init_droplet(R, N / 2, N / 2, 0)
    o.step(steps)
    p, psi = o.get("p"), o.get("psi")
    dp = float(p[psi > 0.99].mean() - p[psi < 0.01].mean())
    R_eff = float(math.sqrt(psi.sum() / math.pi))
    return dict(R=R, W=W, dp=dp, R_eff=R_eff, gamma=0.01)


def contact_angle(theta, R=16.0, nx=96, ny=48, steps=5000):
    W = _W()
    o = _oracle().Oracle(W.params(nx=nx, ny=ny, T_w=0.0, CaE=0.0, R0=R, theta_deg=theta))
    xc, yc = W.sessile_center(nx, R, theta)
    o.init_droplet(R, xc, yc, 0)
    o.step(steps)
    ob = o.observables()
    return dict(theta=theta, height=ob["height"], base_half=ob["R_tr"])


def stefan(Ste=0.1, alpha=0.1, h0=56.0, ny=64, steps=20000, samples=8, alpha_sl=1.0):
    """One-phase Stefan problem: liquid layer at T_m, cold wall below; the
    heat crosses the growing solid layer (diffusivity alpha * alpha_sl)."""
    o = _oracle().Oracle(_W().params(nx=4, ny=ny, rho_sl=1.0, Ste=Ste, alpha_l=alpha,
                                     CaE=0.0, R0=h0, theta_deg=90.0, alpha_sl=alpha_sl))
    o.init_psi(layer_psi(4, ny, h0, 4.0))
    ts, fronts = [], []
    for _ in range(samples):
        o.step(steps // samples)
        ts.append(o.t)
        fronts.append(o.observables()["front"])
    return dict(Ste=Ste, alpha=alpha * alpha_sl, t=ts, front=fronts)


def volume_change(rho_sl, h0=20.0, ny=48, steps=8000):
    o = _oracle().Oracle(_W().params(nx=4, ny=ny, rho_sl=rho_sl, Ste=0.5, alpha_l=0.1,
                                     CaE=0.0, R0=h0, theta_deg=90.0))
    o.init_psi(layer_psi(4, ny, h0, 4.0))
    o.step(steps)
    ob = o.observables()
    return dict(rho_sl=rho_sl, h0=h0, height=ob["height"], frozen=ob["frozen_fraction"])


def deformation(R_sigma, S_eps, CaE=0.2, N=80, R=16.0, steps=5000, presolve=12000):
    """Suspended drop between the electrodes, viscosity and density ratio 1."""
    o = _oracle().Oracle(_W().params(nx=N, ny=N, T_w=0.0, CaE=CaE, R_sigma=R_sigma, S_eps=S_eps,
                                     R0=R, rho_lg=1.0, mu_lg=1.0, k_e=5))
    o.init_droplet(R, N / 2, N / 2, presolve)
    o.step(steps)
    psi = o.get("psi")

    def extent(v):
        idx = np.where(v >= 0.5)[0]
        a, b = idx[0], idx[-1]
        lo = (a - 1) + (0.5 - v[a - 1]) / (v[a] - v[a - 1])
        hi = b + (v[b] - 0.5) / (v[b] - v[b + 1])
        return float(hi - lo)

    L_along = extent(psi[:, N // 2])      # along E (vertical)
    H_perp = extent(psi[N // 2, :])       # perpendicular to E
    return dict(R=R_sigma, S=S_eps, CaE=CaE, D=(L_along - H_perp) / (L_along + H_perp))


def droplet_front(Fo, Ste=0.2, rho_sl=0.9, theta=120.0, alpha_lg=0.2, R=16.0, nx=96, ny=48):
    W = _W()
    p = W.params(nx=nx, ny=ny, Ste=Ste, rho_sl=rho_sl, theta_deg=theta, alpha_lg=alpha_lg,
                 CaE=0.0, R0=R)
    o = _oracle().Oracle(p)
    xc, yc = W.sessile_center(nx, R, theta)
    o.init_droplet(R, xc, yc, 0)
    o.step(int(round(Fo * R * R / p["alpha_l"])))
    ob = o.observables()
    return dict(Fo=ob["Fo"], front_over_R0=ob["front"] / R)


def freezing_time(R_sigma, S_eps, CaE, Ste=0.2, rho_sl=0.9, theta=120.0, alpha_lg=0.2, R=16.0, nx=96, ny=48,
                  every=20, T_g=0.5, Fo_probe=0.3125):
    """Steps until the frozen fraction reaches 0.99, observed every `every`
    steps, with the whole region initially at T_g (T_m = 0, T_w = -1), and
    the droplet's height and contact-line radius at Fo = Fo_probe."""
    W = _W()
    p = W.params(nx=nx, ny=ny, Ste=Ste, rho_sl=rho_sl, theta_deg=theta, alpha_lg=alpha_lg, CaE=CaE,
                 R_sigma=R_sigma, S_eps=S_eps, R0=R, T_init=T_g)
    o = _oracle().Oracle(p)
    xc, yc = W.sessile_center(nx, R, theta)
    o.init_droplet(R, xc, yc, 2000)
    ob = o.observables()
    probe = int(round(Fo_probe * R * R / p["alpha_l"]))
    h_probe = r_probe = None
    while ob["t_fre"] < 0 and o.t < 100000:
        o.step(every)
        ob = o.observables()
        if h_probe is None and o.t >= probe:
            h_probe, r_probe = ob["height"], ob["R_tr"]
    return dict(t_fre=ob["t_fre"], height=ob["height"], R_tr=ob["R_tr"], h_probe=h_probe, R_tr_probe=r_probe)


def shifted_layer(T_m, lib=None, ny=192, h0=20.0, rho_sl=0.9, steps=4000, alpha_lg=5.0):
    """The three-phase Stefan layer of Sec. 4 (liquid on the cold wall under
    gas, closed box) with the temperature origin at T_m: T_w = T_m - 1 and
    T_init = T_m.  A tall, weakly conducting gas column (alpha_l / alpha_g = 5)
    holds most of the compression that the expansion of the freezing liquid
    causes in the closed box.  Frozen fraction after `steps` steps."""
    o = _oracle().Oracle(_W().params(nx=4, ny=ny, rho_sl=rho_sl, Ste=0.5, alpha_l=0.1, CaE=0.0, R0=h0,
                                     theta_deg=90.0, T_m=T_m, T_w=T_m - 1.0, T_init=T_m, alpha_lg=alpha_lg),
                         lib=lib)
    o.init_psi(layer_psi(4, ny, h0, 4.0))
    o.step(steps)
    ob = o.observables()
    return dict(T_m=T_m, frozen=ob["frozen_fraction"])


def shifted_volume_change(T_m, rho_sl=0.9, h0=20.0, ny=48, steps=8000):
    """volume_change with the temperature origin at T_m (T_w = T_m - 1)."""
    o = _oracle().Oracle(_W().params(nx=4, ny=ny, rho_sl=rho_sl, Ste=0.5, alpha_l=0.1, CaE=0.0, R0=h0,
                                     theta_deg=90.0, T_m=T_m, T_w=T_m - 1.0, T_init=T_m))
    o.init_psi(layer_psi(4, ny, h0, 4.0))
    o.step(steps)
    ob = o.observables()
    return dict(rho_sl=rho_sl, h0=h0, T_m=T_m, height=ob["height"], frozen=ob["frozen_fraction"])


def translating_drop(U=0.1, lib=None, N=64, R=12.0, steps=640):
    """A drop (density and viscosity ratio 1, no field, no freezing) carried
    by a uniform flow U along x, periodic in x, in the middle of the channel
    (the wall boundary layers stay away from it for `steps` steps).  The
    state starts at the equilibria of that flow, with psi u of the previous
    step equal to the current one.  Returns the centroid speed over U, the
    ratio of the summed squared x- and y-gradients of psi (1 for an
    isotropic interface) and the mass ratio."""
    W = _W()
    orc = _oracle()
    o = orc.Oracle(W.params(nx=N, ny=N, T_w=0.0, T_m=0.0, T_init=0.0, CaE=0.0, R0=R, rho_lg=1.0, mu_lg=1.0),
                   lib=lib)
    o.init_droplet(R, N / 2, N / 2, 0)
    psi = o.get("psi")
    cx, cy, w = orc.lattice()
    cu = (cx * U)[:, None, None] * np.ones((1, N, N))
    o.set("f", w[:, None, None] * psi[None] * (1 + 3 * cu))                      # Sec. 3.1 equilibrium
    o.set("h", w[:, None, None] * (3 * cu + 4.5 * cu * cu - 1.5 * U * U))         # Sec. 3.2, p = 0, rho = 1
    o.set("psiux", psi * U)
    o.set("psiuy", np.zeros_like(psi))
    m0 = psi.sum()

    def centroid(ps):
        th = 2 * math.pi * np.arange(N) / N
        a = (ps.sum(0) * np.exp(1j * th)).sum()
        return (np.angle(a) % (2 * math.pi)) * N / (2 * math.pi)

    x0 = centroid(psi)
    o.step(steps)
    ps = o.get("psi")
    disp = (centroid(ps) - x0) % N
    gx = (np.roll(ps, -1, 1) - np.roll(ps, 1, 1)) / 2
    gy = np.zeros_like(ps)
    gy[1:-1] = (ps[2:] - ps[:-2]) / 2
    return dict(U=U, speed=disp / (U * steps), aniso=float((gx ** 2).sum() / (gy ** 2).sum()),
                mass=float(ps.sum() / m0))


def mass_conservation(steps=1000):
    """Sessile drop with the field on and no freezing (T_w = T_m)."""
    W = _W()
    p = W.params(nx=128, ny=64, T_w=0.0, k_e=2)
    o = _oracle().Oracle(p)
    xc, yc = W.sessile_center(128, 20.0, 90.0)
    o.init_droplet(20.0, xc, yc, 50)
    m0 = o.observables()["mass"]
    o.step(steps)
    ob = o.observables()
    return dict(m0=m0, m1=ob["mass"], solid=ob["solid"])


def sensitivity(steps=500):
    """Two 128 x 64 sessile runs whose initial f differ by 1e-15 relative."""
    W = _W()
    w = W.plain_fp64_small()
    p = w["params"]
    a, b = _oracle().Oracle(p), _oracle().Oracle(p)
    xc, yc = W.sessile_center(128, 20.0, 90.0)
    a.init_droplet(20.0, xc, yc, 0)
    b.init_droplet(20.0, xc, yc, 0)
    f = b.get("f")
    b.set("f", f * (1 + 1e-15 * W.noise(f.shape, 3)))
    a.step(steps)
    b.step(steps)
    return dict(steps=steps, dpsi=float(np.abs(a.get("psi") - b.get("psi")).max()))


JOBS = {
    "sensitivity": (sensitivity, ()),
    "laplace_10": (laplace, (10.0,)),
    "laplace_14": (laplace, (14.0,)),
    "laplace_18": (laplace, (18.0,)),
    "laplace_14_W5": (laplace, (14.0, 5.0)),
    "laplace_21_W6": (laplace, (21.0, 6.0, 96, 11250)),
    "angle_60": (contact_angle, (60.0,)),
    "angle_90": (contact_angle, (90.0,)),
    "angle_120": (contact_angle, (120.0,)),
    "stefan": (stefan, ()),
    "stefan_solid_diffusivity": (stefan, (0.1, 0.05, 56.0, 64, 20000, 8, 2.0)),
    "volume_0.9": (volume_change, (0.9,)),
    "volume_1.1": (volume_change, (1.1,)),
    "deform_5_2": (deformation, (5.0, 2.0)),
    "deform_2_5": (deformation, (2.0, 5.0)),
    "deform_5_2_N120": (deformation, (5.0, 2.0, 0.2, 120)),
    "deform_5_2_N160": (deformation, (5.0, 2.0, 0.2, 160)),
    "deform_2_5_N160": (deformation, (2.0, 5.0, 0.2, 160)),
    "front_paper": (droplet_front, (0.62,)),
    "mass": (mass_conservation, ()),
    "shift_0": (shifted_layer, (0.0,)),
    "shift_2": (shifted_layer, (2.0,)),
    "volume_0.9_Tm2": (shifted_volume_change, (2.0,)),
    "translate_0.1": (translating_drop, (0.1,)),
    "translate_0.05": (translating_drop, (0.05,)),
    "freeze_off": (freezing_time, (5.0, 2.0, 0.0)),
    "freeze_OB-": (freezing_time, (2.0, 5.0, 1.0)),
    "freeze_PR-": (freezing_time, (5.0, 9.5, 1.0)),
    "freeze_PR+": (freezing_time, (2.0, 0.5, 1.0)),
}


def _run(name):
    fn, args = JOBS[name]
    return name, fn(*args)


def run_all(processes=None):
    import multiprocessing as mp
    import os
    ctx = mp.get_context("spawn")
    procs = processes or min(len(JOBS), max(1, os.cpu_count() or 1))
    # longest jobs first so the pool drains evenly
    order = ["deform_5_2_N160", "deform_2_5_N160", "freeze_off", "freeze_OB-", "freeze_PR-", "freeze_PR+",
             "laplace_21_W6",
             "deform_5_2_N120", "deform_5_2", "deform_2_5", "sensitivity", "laplace_10", "laplace_14", "laplace_18",
             "laplace_14_W5", "angle_60", "angle_90", "angle_120", "front_paper",
             "mass", "stefan", "stefan_solid_diffusivity", "volume_0.9", "volume_1.1",
             "translate_0.1", "translate_0.05", "shift_0", "shift_2", "volume_0.9_Tm2"]
    with ctx.Pool(procs) as pool:
        return dict(pool.map(_run, order, chunksize=1))

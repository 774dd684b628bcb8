"""Parity of the sm_103a library with the FP64 CPU oracle (GPU required).

Fields are compared element by element on the same seeded inputs.  The FP64
library is built without FMA contraction and follows the oracle's operation
order, so its bar is the required tolerance: every stored field within
1e-12 of the oracle's in the max norm relative to the field's largest
magnitude, after up to 1000 steps.  FP32 runs are held to tolerances derived
from single-precision rounding (see test docstrings).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_06657_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STORED = ["f", "h", "g", "l", "fs_prev", "mdot_prev", "Q_prev", "psiux", "psiuy", "p", "S"]
MACROS = ["psi", "fsolid", "T", "phi", "H"]
TOL64 = 1e-12


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_06657_gb300 import lbm as L
    L.load()
    return L


def normwise(a, b, floor=0.0):
    """max|a - b| relative to the field's largest magnitude, or to its
    natural scale where the field is (nearly) zero everywhere."""
    scale = max(float(np.abs(b).max()), floor)
    if scale == 0.0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max()) / scale


def floors(p):
    """Natural scales: a fraction is O(1); T is measured against the imposed
    temperature difference; H against the latent heat; p and h against the
    drop's Laplace pressure; S against rho (1 - rho_s/rho_l) df_s/dt at a
    moving front (1e-3) and psi u against the flow freezing drives (1e-4).  At t = 0, T = T_m and f_s = 0
    everywhere, so max|field| alone would divide last-bit differences of the
    initial tanh profile by ~1e-17."""
    dT = max(p["T_m"] - p["T_w"], 1e-3)
    L = p["cp_l"] * dT / p["Ste"]
    lap = p["gamma"] / p["R0"]          # Laplace pressure of the drop
    return {"psi": 1.0, "fsolid": 1.0, "fs_prev": 1.0, "T": dT, "H": L, "g": L,
            "mdot_prev": 1e-2, "Q_prev": 1e-2, "p": lap, "h": lap, "S": 1e-3,
            "psiux": 1e-4, "psiuy": 1e-4}


def worst(gpu, ref, names=STORED + MACROS):
    fl = floors(gpu.params)
    out = {}
    for n in names:
        out[n] = normwise(gpu.get(n), ref.get(n), fl.get(n, 0.0))
    return out


def pair(L, p, R=None, center=None, presolve=0, psi=None, exact=True):
    """GPU and oracle instances with the same initial state.  exact=True
    hands both the same host psi array (lbm_init_psi), so the FP64 runs start
    from identical bits; exact=False uses each side's own droplet initialiser
    (tanh evaluated by CUDA and by libm: last-bit differences)."""
    g, o = L.Simulation(p), oracle.Oracle(p)
    if psi is None and exact:
        if center is None:
            center = W.sessile_center(p["nx"], R, p["theta_deg"])
        psi = W.droplet_psi(p["nx"], p["ny"], R, center[0], center[1], p["W"])
    if psi is not None:
        g.init_psi(psi, presolve)
        o.init_psi(psi, presolve)
    else:
        if center is None:
            center = W.sessile_center(p["nx"], R, p["theta_deg"])
        g.init_droplet(R, center[0], center[1], presolve)
        o.init_droplet(R, center[0], center[1], presolve)
    return g, o


def assert_fp64(errs, tol=TOL64):
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"normwise differences above {tol}: {bad}"


# --------------------------------------------------------------------------
# FP64 step parity
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,R,theta", [(8, 6, 3.0, 90.0), (16, 8, 5.0, 60.0), (4, 3, 2.0, 120.0),
                                           (50, 21, 9.0, 110.0)])
def test_fp64_matches_oracle_step_by_step(lbm, nx, ny, R, theta):
    """Tiny and ragged lattices (tiles of 32 x 8 with partial tails), the
    field and the cold wall on, after 1, 2 and 10 steps."""
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=theta, precision=W.FP64)
    g, o = pair(lbm, p, R)
    assert_fp64(worst(g, o), 0.0)              # identical initial state
    done = 0
    for n in (1, 2, 10):
        g.step(n - done)
        o.step(n - done)
        done = n
        assert_fp64(worst(g, o))


@pytest.mark.parametrize("nx,ny", [(8, 6), (16, 8), (37, 19)])
def test_fp64_matches_oracle_after_1000_steps(lbm, nx, ny):
    """Required bar: fields within 1e-12 (normwise) after 1000 steps, with
    two potential sweeps per step and a pre-solve."""
    R = 0.35 * ny
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=75.0, precision=W.FP64, k_e=2, Ste=0.3)
    g, o = pair(lbm, p, R, presolve=10)
    g.step(1000)
    o.step(1000)
    assert_fp64(worst(g, o))


def test_droplet_initialisers_agree(lbm):
    """lbm_init_droplet (tanh on the GPU) against the oracle's initialiser
    (libm tanh): the initial states differ only in the last bits."""
    p = W.params(nx=96, ny=48, R0=16.0, theta_deg=70.0, precision=W.FP64, k_e=1)
    g, o = pair(lbm, p, 16.0, presolve=25, exact=False)
    assert_fp64(worst(g, o), 1e-15)
    g.step(5)
    o.step(5)
    assert_fp64(worst(g, o))


def test_presolve_to_a_tolerance(lbm):
    """lbm_presolve sweeps the potential until phi changes by less than
    tol x |phi_top - phi_bot| over one sweep (checked every 64 sweeps).  The
    linear potential of the initial state is already the fixed point of a
    drop-free lattice; with a droplet, the sweep count it reports reproduces
    the oracle's fixed-count pre-solve, and a cap below it gives the
    NOT_CONVERGED warning with the count and residual reached."""
    p = W.params(nx=32, ny=16, R0=5.0, precision=W.FP64)
    s = lbm.Simulation(p)
    s.init_psi(np.zeros((16, 32)), 0)
    r = s.presolve(1e-12, 10000)
    assert r["converged"] and r["sweeps"] == 64 and r["residual"] < 1e-12, r

    p = W.params(nx=40, ny=20, R0=7.0, theta_deg=100.0, precision=W.FP64)
    xc, yc = W.sessile_center(40, 7.0, 100.0)
    psi0 = W.droplet_psi(40, 20, 7.0, xc, yc, p["W"])
    g = lbm.Simulation(p)
    g.init_psi(psi0, 0)
    r = g.presolve(1e-9, 200000)
    assert r["converged"] and r["residual"] < 1e-9 and r["sweeps"] % 64 == 0, r
    ref = oracle.Oracle(p)
    ref.init_psi(psi0, r["sweeps"])
    for name in ("l", "phi"):
        a, b = g.get(name), ref.get(name)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), name
    h = lbm.Simulation(p)
    h.init_psi(psi0, 0)
    w = h.presolve(1e-9, 128)
    assert not w["converged"] and w["sweeps"] == 128 and w["residual"] >= 1e-9, w
    f32 = lbm.Simulation(W.params(nx=40, ny=20, R0=7.0, theta_deg=100.0, precision=W.FP32))
    f32.init_psi(psi0, 0)
    r32 = f32.presolve(1e-5, 200000)
    assert r32["converged"] and r32["sweeps"] <= r["sweeps"], r32
    # half storage: the sweeps round stochastically (to nearest they stalled
    # 1.2e-2 of the range short of the solution), so phi reaches the FP64
    # solution to 2e-4 of the range, while the rounding noise keeps the
    # per-sweep change near 4e-4: a tighter tolerance ends with the warning
    f16 = lbm.Simulation(W.params(nx=40, ny=20, R0=7.0, theta_deg=100.0, precision=W.FP16S))
    f16.init_psi(psi0, 0)
    r16 = f16.presolve(1e-7, 20000)
    assert not r16["converged"] and r16["sweeps"] == 20000 and r16["residual"] > 1e-5, r16
    assert np.abs(f16.get("phi") - g.get("phi")).max() <= 1e-3 * np.abs(g.get("phi")).max()


def test_fp64_matches_oracle_on_the_128x64_case(lbm):
    """The 128 x 64 sessile case (R = 20, theta = 90, CaE = 0.2, S = 2,
    R = 5, Ste = 0.5), 1000 steps; observables agree too."""
    w = W.plain_fp64_small()
    p = w["params"]
    g, o = pair(lbm, p, w["R"])
    g.step(1000)
    o.step(1000)
    assert_fp64(worst(g, o))
    og, oo = g.observables(), o.observables()
    for k in ("mass", "enthalpy", "solid", "frozen_fraction"):
        assert abs(og[k] - oo[k]) <= 1e-12 * max(abs(oo[k]), 1.0), k
    assert abs(og["charge"] - oo["charge"]) <= 1e-10 * max(abs(oo["charge"]), 1e-3)
    for k in ("height", "width", "aspect", "R_tr", "front"):
        assert abs(og[k] - oo[k]) <= 1e-9 * max(abs(oo[k]), 1.0), k
    assert og["step"] == oo["step"] == 1000 and og["status"] == 0
    for k in ("Pe", "Qdot"):
        assert oo[k] != 0.0, k
        assert abs(og[k] - oo[k]) <= 1e-12 * abs(oo[k]), k
    qg, qo = g.substrate_heat_flux(), o.heat_flux()
    assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()


def test_observables_over_uneven_reduction_groups(lbm):
    """A 300 x 100 lattice has 130 reduction blocks: four full groups of 32
    and a last group of 2, so both levels of the observables' finish run
    with a partial group.  FP64 sums to 1e-12 of the oracle's, geometry to
    1e-9, after 60 steps from a droplet off the centre."""
    p = W.params(nx=300, ny=100, R0=30.0, theta_deg=70.0, precision=W.FP64)
    g, o = pair(lbm, p, 30.0, center=(110.0, W.sessile_center(300, 30.0, 70.0)[1]))
    g.step(60)
    o.step(60)
    og, oo = g.observables(), o.observables()
    for k in ("mass", "enthalpy", "solid", "frozen_fraction", "Pe", "Qdot"):
        assert abs(og[k] - oo[k]) <= 1e-12 * max(abs(oo[k]), 1e-30), k
    assert abs(og["charge"] - oo["charge"]) <= 1e-10 * max(abs(oo["charge"]), 1e-3)
    for k in ("height", "width", "aspect", "R_tr", "front"):
        assert abs(og[k] - oo[k]) <= 1e-9 * max(abs(oo[k]), 1.0), k


@pytest.mark.parametrize("substance", ["water", "hexadecane"])
def test_fp64_table1_property_sets(lbm, substance):
    """Table 1 property sets (solid diffusivity and heat capacity differ from
    the liquid's, rho_s/rho_l = 0.918 or 1.076, theta = 87): fields, Pe, Qdot
    and the substrate heat-flux profile match the oracle after 300 steps on a
    ragged 70 x 36 lattice."""
    case = W.table1_case(substance, precision=W.FP64, nx=70, ny=36)
    p = case["params"]
    g, o = pair(lbm, p, case["R"])
    g.step(300)
    o.step(300)
    assert_fp64(worst(g, o))
    og, oo = g.observables(), o.observables()
    assert oo["frozen_fraction"] > 0.01
    for k in ("mass", "enthalpy", "solid", "Pe", "Qdot"):
        assert abs(og[k] - oo[k]) <= 1e-12 * max(abs(oo[k]), 1e-30), k
    qg, qo = g.substrate_heat_flux(), o.heat_flux()
    assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()


@pytest.mark.parametrize("prec,tol_q,tol_pe", [(W.FP32, 1e-4, 1e-2), (W.FP16S, 3e-2, 0.25)],
                         ids=["fp32", "fp16s"])
def test_single_precision_extra_observables(lbm, prec, tol_q, tol_pe):
    """Pe and the substrate heat flux of the single-precision paths against
    the FP64 oracle on the 128 x 64 case after 200 steps.  FP32: the heat
    flux to 1e-4 of its largest magnitude, Qdot to 1e-4 and Pe (a ratio of
    small velocities) to 1e-2 relative.  Half storage keeps 11 significant
    bits and rounds stochastically, and the flux is a difference of nearby
    temperatures: 3e-2, and 0.25 for Pe."""
    w = W.plain_fp64_small()
    p = dict(w["params"], precision=prec)
    g, o = pair(lbm, p, w["R"])
    g.step(200)
    o.step(200)
    og, oo = g.observables(), o.observables()
    qg, qo = g.substrate_heat_flux(), o.heat_flux()
    eq = np.abs(qg - qo).max() / np.abs(qo).max()
    assert eq <= tol_q, eq
    assert abs(og["Qdot"] / oo["Qdot"] - 1) < tol_q, (og["Qdot"], oo["Qdot"])
    assert abs(og["Pe"] / oo["Pe"] - 1) < tol_pe, (og["Pe"], oo["Pe"])


@pytest.mark.parametrize("k_e", [1, 3])
def test_fp64_parity_from_perturbed_states(lbm, k_e):
    """Seeded noise on every stored field (populations, the lagged solid
    fraction, mass source, enthalpy source, psi u, p, S) drives cells into
    every branch of the enthalpy inversion and the force terms."""
    nx, ny, R = 40, 24, 8.0
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=100.0, precision=W.FP64, k_e=k_e)
    g, o = pair(lbm, p, R)
    o.step(30)
    seed = 11
    for name, scale in [("f", 0.02), ("h", 1e-3), ("g", 0.05), ("l", 1e-3), ("fs_prev", 0.5),
                        ("mdot_prev", 0.01), ("Q_prev", 0.01), ("psiux", 1e-3), ("psiuy", 1e-3),
                        ("p", 1e-3), ("S", 1e-3)]:
        v = o.get(name)
        v = v + W.noise(v.shape, seed, scale)
        seed += 1
        o.set(name, v)
        g.set(name, v)
    assert_fp64(worst(g, o), 0.0 + 1e-15)
    g.step(3)
    o.step(3)
    assert_fp64(worst(g, o))


def test_fp64_full_size_production_lattice(lbm):
    """512 x 256, R = 80, in the launch configuration the benchmark times:
    every field of every cell after 3 steps (the oracle runs a full step of
    this size in a fraction of a second)."""
    w = W.production(precision=W.FP64)
    p = w["params"]
    g, o = pair(lbm, p, w["R"])
    g.step(3)
    o.step(3)
    assert_fp64(worst(g, o))


def test_fp64_full_size_precision_lattice(lbm):
    """1024 x 512, R = 160, theta = 60, PR+ field (the largest lattice the
    benchmark times), in its launch configuration: every field of every cell
    after 2 steps against the oracle."""
    w = W.precision_case(W.FP64)
    p = w["params"]
    g, o = pair(lbm, p, w["R"])
    g.step(2)
    o.step(2)
    assert_fp64(worst(g, o))


def test_fp32_full_size_precision_lattice_observables(lbm):
    """1024 x 512 FP32 in the benchmark's launch configuration against the
    FP64 oracle after 5 steps: conserved sums to 1e-5 relative, interface
    geometry to 1e-3 lattice units."""
    w = W.precision_case(W.FP32)
    p = w["params"]
    g, o = pair(lbm, p, w["R"])
    g.step(5)
    o.step(5)
    og, oo = g.observables(), o.observables()
    for k in ("mass", "enthalpy"):
        assert abs(og[k] / oo[k] - 1) < 1e-5, k
    for k in ("height", "width", "R_tr"):
        assert abs(og[k] - oo[k]) < 1e-3, k


@pytest.mark.parametrize("nx,ny", [(4, 3), (37, 19), (64, 32), (100, 45), (33, 9)])
def test_tile_heights_agree_bitwise(lbm, nx, ny):
    """The in-place step reads its halo from the neighbour tiles' populations
    or, once a neighbour has started to overwrite them, from the macros that
    neighbour published; which route a halo cell takes depends on the tile
    shape and on scheduling, and both must give the same FP64 bits.  Every
    tile height, on ragged and tiny lattices (one tile column, a wrap-around
    lane), over an even and an odd number of steps (both layouts)."""
    R = 0.3 * min(nx, 2 * ny)
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=105.0, precision=W.FP64, k_e=2)
    xc, yc = W.sessile_center(nx, R, 105.0)
    psi = W.droplet_psi(nx, ny, R, xc, yc, p["W"])
    ref = lbm.Simulation(p)
    ref.configure(lbm.STEP_DIRECT, 8)
    ref.init_psi(psi, 4)
    for n in (40, 1):
        ref.step(n)
        want = {k: ref.get(k) for k in STORED}
        for rows in (4, 16):
            s = lbm.Simulation(p)
            s.configure(lbm.STEP_DIRECT, rows)
            s.init_psi(psi, 4)
            s.step(ref.t)
            for k in STORED:
                assert np.array_equal(s.get(k), want[k]), (rows, n, k)


@pytest.mark.parametrize("prec", [W.FP32, W.FP16S])
def test_single_precision_runs_are_reproducible(lbm, prec):
    """Whether a halo cell's macros come from its populations or from the
    record its owner published depends on scheduling; in single precision
    both routes round every operation separately (no FMA fusion), so two
    runs from the same state give the same bits, alone and batched, over a
    freezing front and a lattice of many tiles with a ragged edge."""
    nx, ny, R = 250, 126, 60.0
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=95.0, CaE=0.2, precision=prec)
    xc, yc = W.sessile_center(nx, R, 95.0)
    psi = W.droplet_psi(nx, ny, R, xc, yc, p["W"])
    runs = []
    for _ in range(2):
        s = lbm.Simulation(p)
        s.configure(lbm.STEP_DIRECT, 4)
        s.init_psi(psi, 3)
        s.step(301)
        runs.append({k: s.get(k) for k in STORED})
    for k in STORED:
        assert np.array_equal(runs[0][k], runs[1][k]), k
    batches = []
    for _ in range(2):
        sims = []
        for th in (95.0, 120.0):
            q = W.params(nx=nx, ny=ny, R0=R, theta_deg=th, CaE=0.2, precision=prec)
            s = lbm.Simulation(q)
            s.init_droplet(R, *W.sessile_center(nx, R, th), 3)
            sims.append(s)
        lbm.Batch(sims, tile_rows=4).step(301)
        batches.append([{k: s.get(k) for k in STORED} for s in sims])
    for m0, m1 in zip(*batches):
        for k in STORED:
            assert np.array_equal(m0[k], m1[k]), k


def test_graph_replay_and_single_launches_agree_bitwise(lbm):
    """lbm_step(64) replays a captured graph; 64 single steps must give the
    same bits."""
    p = W.params(nx=64, ny=32, R0=10.0, precision=W.FP64, k_e=2)
    xc, yc = W.sessile_center(64, 10.0, 90.0)
    a, b = lbm.Simulation(p), lbm.Simulation(p)
    a.init_droplet(10.0, xc, yc, 5)
    b.init_droplet(10.0, xc, yc, 5)
    a.step(64)
    for _ in range(64):
        b.step(1)
    for n in STORED:
        assert np.array_equal(a.get(n), b.get(n)), n
    assert a.t == b.t == 64


def test_streamed_observables_equal_synchronous_ones(lbm):
    """lbm_observables_to_host enqueues the reduction and its copy into
    page-locked host memory without waiting; after lbm_sync every record
    equals what lbm_observables returns at the same step."""
    import ctypes
    import torch
    p = W.params(nx=128, ny=64, R0=20.0, precision=W.FP32)
    xc, yc = W.sessile_center(128, 20.0, 90.0)
    a, b = lbm.Simulation(p), lbm.Simulation(p)
    a.init_droplet(20.0, xc, yc, 0)
    b.init_droplet(20.0, xc, yc, 0)
    n, sz = 6, ctypes.sizeof(lbm.Obs)
    buf = torch.zeros(n * sz, dtype=torch.uint8, pin_memory=True)
    want = []
    for i in range(n):
        a.step(10)
        a.observables_to_host(buf.data_ptr() + i * sz)
        b.step(10)
        want.append(b.observables())
    a.sync()
    got = [lbm.Obs.from_address(buf.data_ptr() + i * sz).as_dict() for i in range(n)]
    assert got == want
    assert [g["step"] for g in got] == [10 * (i + 1) for i in range(n)]


# --------------------------------------------------------------------------
# Batched form: same bits as stepping alone
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tile", [(W.FP64, 0), (W.FP32, 8), (W.FP32, 0), (W.FP16S, 4)])
def test_batch_equals_members_stepped_alone(lbm, prec, tile):
    """Uneven members, a member that starts at the other parity.  FP64
    results are bitwise those of stepping alone whatever the tile shape and
    kernel form (no FMA contraction, same operation order).  In FP32 the
    members alone use the batch's tile height; the batched kernel and the
    single-instance kernel may still round differently (FMA contraction
    in different kernel bodies): the fields must agree to 1e-3 after 20
    steps (max norm with natural-scale floors), before last-bit differences
    grow at the freezing front (the source S is a difference of consecutive
    f_s and amplifies them most), and after 300 steps the observables to
    1e-4, the accuracy bar for single precision.  Half
    storage uses the same rounding
    bits in both forms, but a last-bit difference before rounding moves a
    stored value by a whole half spacing: its bar is the observables, to
    1e-3."""
    cases = [(96, 48, 15.0, 80.0, 0.1, 2.0, 5.0), (64, 32, 10.0, 110.0, 0.4, 0.5, 2.0),
             (37, 21, 6.0, 95.0, 0.0, 5.0, 9.5)]
    sims, alone = [], []
    for nx, ny, R, th, ca, rs, se in cases:
        p = W.params(nx=nx, ny=ny, R0=R, theta_deg=th, CaE=ca, R_sigma=rs, S_eps=se, precision=prec)
        xc, yc = W.sessile_center(nx, R, th)
        for lst in (sims, alone):
            s = lbm.Simulation(p)
            s.init_droplet(R, xc, yc, 3)
            lst.append(s)
    alone[1].step(1)          # members may start at different parities
    sims[1].step(1)
    b = lbm.Batch(sims, tile_rows=tile)
    assert b.tile_rows in (4, 8, 16)
    if prec != W.FP64:        # same tile height, so the same arithmetic per tile
        for s in alone:
            s.configure(lbm.STEP_DIRECT, b.tile_rows)
    n = 45 if prec == W.FP64 else 20
    b.step(n)                # graphs of 32 steps + single launches
    for s in alone:
        s.step(n)
    for s, a in zip(sims, alone):
        assert s.t == a.t
        fl = floors(s.params)
        for name in STORED:
            if prec == W.FP64:
                assert np.array_equal(s.get(name), a.get(name)), name
            elif prec == W.FP32:
                assert normwise(s.get(name), a.get(name), fl.get(name, 0.0)) <= 1e-3, name
    if prec == W.FP64:
        return
    # single precision: the two kernels' last-bit differences grow at the
    # freezing front (a cell crosses the solidus a step apart); the bar
    # over the longer horizon is on the observables
    b.step(280)
    for s in alone:
        s.step(280)
    for s, a in zip(sims, alone):
        assert s.t == a.t
        if prec != W.FP64:
            tol = 1e-4 if prec == W.FP32 else 1e-3
            os_, oa = s.observables(), a.observables()
            # the enthalpy sum nearly cancels (cold gas and ice below zero,
            # liquid holding its latent heat above): it is measured against
            # the droplet's latent heat, L times its mass, not its own size
            # (half storage keeps 11 bits of every enthalpy population and
            # rounds them stochastically: once the two kernels' single-
            # precision bits differ, the sums drift apart by about 1e-3 of
            # that latent heat in 300 steps, so its enthalpy bar is 3e-3)
            latent = s.params["cp_l"] * (s.params["T_m"] - s.params["T_w"]) / s.params["Ste"] * oa["mass"]
            for k in ("mass", "enthalpy", "frozen_fraction", "height", "width", "aspect"):
                scale = max(abs(oa[k]), latent if k == "enthalpy" else 1.0)
                t_k = 3e-3 if (k == "enthalpy" and prec == W.FP16S) else tol
                assert abs(os_[k] - oa[k]) <= t_k * scale, k


def test_batch_in_l2_groups_equals_members_stepped_alone(lbm):
    """Members whose combined state exceeds half of L2 are stepped in
    L2-sized groups, each group all n steps at a time; FP64 results are the
    bits of stepping every member alone."""
    sims, alone = [], []
    for th, ca in ((80.0, 0.2), (100.0, 0.0), (95.0, 0.4)):
        p = W.params(nx=384, ny=192, R0=60.0, theta_deg=th, CaE=ca, precision=W.FP64)
        xc, yc = W.sessile_center(384, 60.0, th)
        psi = W.droplet_psi(384, 192, 60.0, xc, yc, p["W"])
        for lst in (sims, alone):
            s = lbm.Simulation(p)
            s.init_psi(psi, 2)
            lst.append(s)
    b = lbm.Batch(sims, tile_rows=8)
    b.step(40)
    b.step(3)                # short call: one launch per step over all members
    for s in alone:
        s.step(43)
    for s, a in zip(sims, alone):
        assert s.t == a.t == 43
        for n in STORED:
            assert np.array_equal(s.get(n), a.get(n)), n


# --------------------------------------------------------------------------
# Snapshots, errors, divergence
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [W.FP64, W.FP32, W.FP16S])
@pytest.mark.parametrize("at", [7, 8])
def test_snapshot_resume_is_bitwise(lbm, prec, at):
    """A snapshot taken in either layout phase of the in-place streaming
    (after an odd or an even number of steps, k_e = 2 so l keeps its own
    phase) resumes bit for bit; its populations are stored in the natural
    layout (field by field equal to lbm_get_field)."""
    p = W.params(nx=48, ny=24, R0=8.0, precision=prec, k_e=2)
    xc, yc = W.sessile_center(48, 8.0, 90.0)
    a = lbm.Simulation(p)
    a.init_droplet(8.0, xc, yc, 0)
    a.step(at)
    snap = a.export_state()
    f_nat = a.get("f")
    a.step(20)
    ref = {n: a.get(n) for n in STORED}
    b = lbm.Simulation(p)
    b.import_state(snap)
    assert b.t == at
    assert np.array_equal(b.get("f"), f_nat)
    b.step(20)
    for n in STORED:
        assert np.array_equal(b.get(n), ref[n]), n


def _obs_close(got, want, rel):
    """Observables equal up to the grouping of the FP64 sums: counters,
    status and the crossing-based lengths exactly, sums to `rel`."""
    for k, v in want.items():
        g = got[k]
        if k in ("mass", "enthalpy", "solid", "charge", "frozen_fraction", "Pe", "Qdot", "Fo_fre", "Fo"):
            assert abs(g - v) <= rel * max(abs(v), 1e-300) or g == v, (k, g, v)
        else:
            assert g == v, (k, g, v)


@pytest.mark.parametrize("prec,nx,ny,tile,k_e", [(W.FP64, 37, 19, 8, 1), (W.FP64, 64, 32, 4, 2),
                                                 (W.FP64, 40, 3, 8, 1), (W.FP32, 128, 64, 4, 1),
                                                 (W.FP16S, 96, 48, 4, 1), (W.FP32, 100, 45, 16, 1)])
def test_observation_fused_into_the_next_step(lbm, prec, nx, ny, tile, k_e):
    """lbm_observables_deferred + lbm_step: the first step's kernel also
    reduces the observables of the state it reads.  They equal what
    lbm_observables returns for that state (FP64 sums to 1e-13: the step's
    tiles group them differently), and the state after the steps equals a
    plain run's bit for bit, over several observations, across graph
    replays and with extra potential sweeps."""
    p = W.params(nx=nx, ny=ny, R0=ny / 3.0 + 1.0, precision=prec, k_e=k_e)
    xc, yc = W.sessile_center(nx, ny / 3.0 + 1.0, 90.0)
    a, b = lbm.Simulation(p), lbm.Simulation(p)
    for s in (a, b):
        s.configure(lbm.STEP_DIRECT, tile)
        s.init_droplet(ny / 3.0 + 1.0, xc, yc, 2)
        s.step(5)
    rel = 1e-13 if prec == W.FP64 else 1e-6
    for n in (1, 40, 3):
        want = b.observables()
        b.step(n)
        a.observables_deferred()
        a.step(n)
        _obs_close(a.observables_fetch(), want, rel)
    for name in STORED:
        assert np.array_equal(a.get(name), b.get(name)), name


def test_deferred_observation_runs_before_other_calls(lbm):
    """A deferred observation that no step takes runs on its own before the
    next call's work: a field read, a state import, a synchronisation, or
    the next request; with a host address it lands there."""
    import ctypes
    import torch
    p = W.params(nx=48, ny=24, R0=8.0, precision=W.FP64)
    xc, yc = W.sessile_center(48, 8.0, 90.0)
    a = lbm.Simulation(p)
    a.init_droplet(8.0, xc, yc, 0)
    a.step(6)
    want = a.observables()
    snap = a.export_state()
    a.observables_deferred()
    psi = a.get("psi")                       # runs the observation first
    _obs_close(a.observables_fetch(), want, 1e-15)
    a.observables_deferred()
    a.import_state(snap)                     # same state: same observables
    _obs_close(a.observables_fetch(), want, 1e-15)
    buf = torch.zeros(2 * ctypes.sizeof(lbm.Obs), dtype=torch.uint8, pin_memory=True)
    a.observables_deferred(buf.data_ptr())
    a.observables_deferred(buf.data_ptr() + ctypes.sizeof(lbm.Obs))   # runs the first one
    a.sync()                                                           # runs the second one
    for i in range(2):
        _obs_close(lbm.Obs.from_address(buf.data_ptr() + i * ctypes.sizeof(lbm.Obs)).as_dict(), want, 1e-15)
    assert np.array_equal(psi, a.get("psi"))


def test_deferred_observation_of_a_batch_member(lbm):
    """A batch step first runs a member's deferred observation on its own:
    the batch overwrites the state it refers to."""
    p = W.params(nx=64, ny=32, R0=10.0, precision=W.FP64)
    xc, yc = W.sessile_center(64, 10.0, 90.0)
    sims = [lbm.Simulation(p) for _ in range(2)]
    for s in sims:
        s.init_droplet(10.0, xc, yc, 0)
        s.step(3)
    want = sims[0].observables()
    sims[0].observables_deferred()
    b = lbm.Batch(sims, tile_rows=8)
    b.step(2)
    _obs_close(sims[0].observables_fetch(), want, 1e-15)
    assert sims[0].t == 5


def test_back_to_back_imports_from_pinned_memory(lbm):
    """Imports are copied on a private stream into two alternating device
    buffers while the handle's stream still steps the previous state: three
    imports in a row, each followed by steps and a streamed observation,
    give the observables of uninterrupted runs from those snapshots."""
    import ctypes
    import torch
    p = W.params(nx=96, ny=48, R0=15.0, precision=W.FP32)
    xc, yc = W.sessile_center(96, 15.0, 90.0)
    a = lbm.Simulation(p)
    a.init_droplet(15.0, xc, yc, 0)
    n = a.state_bytes()
    s1 = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    s2 = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    a.step(7)
    a.export_state(s1.numpy())
    a.step(5)
    ref1 = a.observables()
    a.step(15)
    a.export_state(s2.numpy())
    a.step(5)
    ref2 = a.observables()
    b = lbm.Simulation(p)
    b.init_droplet(15.0, xc, yc, 0)
    b.step(3)
    sz = ctypes.sizeof(lbm.Obs)
    out = torch.zeros(3 * sz, dtype=torch.uint8, pin_memory=True)
    for i, snap in enumerate((s1, s2, s1)):
        b.import_state(snap.data_ptr())
        b.step(5)
        b.observables_to_host(out.data_ptr() + i * sz)
    b.sync()
    got = [lbm.Obs.from_address(out.data_ptr() + i * sz).as_dict() for i in range(3)]
    assert got == [ref1, ref2, ref1]


def test_error_codes(lbm):
    p = W.params(nx=16, ny=8, R0=4.0)
    s = lbm.Simulation(p)
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == lbm.ERR_STATE
    with pytest.raises(lbm.LBMError) as e:
        s.init_droplet(-1.0, 8, 0, 0)
    assert e.value.code == lbm.ERR_BADPARAM
    with pytest.raises(lbm.LBMError) as e:
        s.substrate_heat_flux()
    assert e.value.code == lbm.ERR_STATE
    s.init_droplet(4.0, 8.0, -0.5, 0)
    with pytest.raises(lbm.LBMError) as e:
        s.set("psi", np.zeros((8, 16)))
    assert e.value.code == lbm.ERR_BADPARAM
    with pytest.raises(lbm.LBMError) as e:
        s.configure(7, 4)                  # no such step variant
    assert e.value.code == lbm.ERR_BADPARAM
    with pytest.raises(lbm.LBMError) as e:
        s.configure(lbm.STEP_DIRECT, 6)    # no such tile height
    assert e.value.code == lbm.ERR_BADPARAM
    thin = lbm.Simulation(W.params(nx=16, ny=2, R0=1.0))
    thin.init_psi(np.zeros((2, 16)))
    with pytest.raises(lbm.LBMError) as e:
        thin.substrate_heat_flux()
    assert e.value.code == lbm.ERR_BADPARAM
    assert thin.observables()["Qdot"] == 0.0


def test_divergence_is_reported_and_stops_stepping(lbm):
    """A non-finite population planted on the host is detected by the
    observables reduction; the handle then refuses to step."""
    p = W.params(nx=32, ny=16, R0=6.0)
    s = lbm.Simulation(p)
    s.init_droplet(6.0, 16.0, -0.5, 0)
    s.step(2)
    f = s.get("f")
    f[0, 3, 5] = np.nan
    s.set("f", f)
    o = s.observables()
    assert o["status"] == lbm.ERR_DIVERGED
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == lbm.ERR_DIVERGED


# --------------------------------------------------------------------------
# FP32 against the FP64 oracle
# --------------------------------------------------------------------------

def test_fp32_fields_track_the_oracle_over_a_short_horizon(lbm):
    """FP32 storage and arithmetic against the FP64 oracle, 20 steps of the
    128 x 64 case: unit roundoff 6e-8 and a few hundred operations per cell
    update give ~1e-6 per step; bar 1e-4 (normwise, natural-scale floors)
    on every stored field.  Over long horizons the scheme's sensitivity near
    the wall on the droplet axis grows last-bit differences, so long FP32
    runs are assessed on observables (next tests)."""
    w = W.plain_fp64_small()
    p = dict(w["params"], precision=W.FP32)
    g, o = pair(lbm, p, w["R"])
    g.step(20)
    o.step(20)
    errs = worst(g, o)
    for k, v in errs.items():
        assert v <= 1e-4, (k, v)


def test_fp32_observables_over_2000_steps(lbm):
    """Accuracy bar for FP32 runs: frozen fraction within 0.5 % and aspect
    ratio within 1 % of the FP64 oracle (128 x 64 case, 2000 steps)."""
    w = W.plain_fp64_small()
    p = dict(w["params"], precision=W.FP32)
    g, o = pair(lbm, p, w["R"])
    g.step(2000)
    o.step(2000)
    og, oo = g.observables(), o.observables()
    assert abs(og["frozen_fraction"] / oo["frozen_fraction"] - 1) < 0.005
    assert abs(og["aspect"] / oo["aspect"] - 1) < 0.01
    assert abs(og["mass"] / oo["mass"] - 1) < 1e-4


def test_fp32_full_size_observables(lbm):
    """512 x 256 FP32 against the FP64 oracle after 20 steps: conserved sums
    to 1e-5 relative, interface geometry to 1e-3 lattice units."""
    w = W.production(precision=W.FP32)
    p = w["params"]
    g, o = pair(lbm, p, w["R"])
    g.step(20)
    o.step(20)
    og, oo = g.observables(), o.observables()
    for k in ("mass", "enthalpy"):
        assert abs(og[k] / oo[k] - 1) < 1e-5, k
    assert abs(og["solid"] - oo["solid"]) <= 1e-4 * oo["mass"]
    for k in ("height", "width", "R_tr"):
        assert abs(og[k] - oo[k]) < 1e-3, k

"""Parity at full size, in the launch configuration bench.py times (autotuned
pair-kernel shape, automatic cell size), on sampled particles that the oracle
computes one by one; plus properties that hold at any size.

Cases: the 0.9 M-particle dam break with obstacle (dp = 0.01 m) in both forms,
the same geometry at dp = 0.005 m (6.3 M particles, mixed), the 8 M-particle
wall-impact tank (dp = 0.0025 m, mixed), the obstacle case at dp = 0.0075 m
with the paper's h and c0 (2.0 M particles, mixed) and the 64-instance alpha
sweep (mixed, batched).  Mixed vs FP64: wave heights within 2 % of the column
height over 1 s of the small dam break.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import load_state, normwise, oracle_case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
MIXED_TOL = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _jittered_full(c, seed):
    case = oracle_case(c)
    st = oracle.scene(case)
    f = st.type == oracle.FLUID
    r, u, rho = wl.perturb(st.r, st.u, st.rho, f, seed, pos_sigma=0.1 * c.dp, vel_sigma=0.2, rho_sigma=1.0)
    return case, oracle.State(r, u, rho, st.type)


def _sample(n, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(n, k), replace=False)).astype(np.int64)


def _check_sample(sim, case, st, sel, tol, exact_counts, fluid_counts_only=False):
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives_subset(case, st, sel)
    assert normwise(drho[sel], o[0]) <= tol
    assert normwise(acc[sel], o[1]) <= tol
    assert normwise(mu[sel], o[2]) <= tol
    if exact_counts:
        assert np.array_equal(nn[sel], o[3])
    else:
        # at h = 1.5 dp the unjittered boundary lattice has pairs at exactly 2h,
        # which FP32 offsets put either side (their terms vanish there)
        m = st.type[sel] == oracle.FLUID if fluid_counts_only else np.ones(len(sel), bool)
        assert np.mean(np.abs(nn[sel][m] - o[3][m])) < 0.05
    # any-size property: the pair parts of m a cancel over all particles
    pair = acc.copy()
    fl = st.type == oracle.FLUID
    pair[fl & (nn >= 0), 2] += 9.81
    assert np.abs(pair.sum(axis=0)).max() <= 1e-6 * np.abs(pair).sum()


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
def test_obstacle_case_dp001_sampled(prec):
    c = wl.obstacle_dambreak()
    case, st = _jittered_full(c, 31)
    sim = sph.Simulation(c, precision=prec)
    load_state(sim, st)
    if prec == sph.MIXED:
        sim.autotune(1)
    sel = _sample(st.n, 3000, 1)
    _check_sample(sim, case, st, sel, FP64_TOL if prec == sph.FP64 else MIXED_TOL, prec == sph.FP64)


@pytest.mark.parametrize("name", ["dambreak_obstacle_dp0.005", "wall_impact_dp0.0025",
                                  "dambreak_obstacle_dp0.0075_paper"])
def test_large_cases_mixed_sampled(name):
    c = wl.by_name(name)
    case, st = _jittered_full(c, 37)
    sim = sph.Simulation(c, precision=sph.MIXED)
    load_state(sim, st)
    sim.autotune(1)
    sel = _sample(st.n, 2000, 2)
    _check_sample(sim, case, st, sel, MIXED_TOL, False, fluid_counts_only=name.endswith("_paper"))
    # and it steps stably for a few adaptive steps
    sim.step(0.0, 5)
    sim.sync()


def test_alpha_sweep_batch_sampled():
    cases = wl.alpha_sweep(64, seed=2306)
    sim = sph.Simulation(cases, precision=sph.MIXED, batch=True)
    sim.autotune(1)
    g = sim.get_state()
    drho, acc, mu, nn = sim.derivatives()
    for k in (0, 17, 63):
        c = cases[k]
        case = oracle_case(c)
        n = int(sim.counts(k)[3])
        off_k = int(sum(sim.counts(j)[3] for j in range(k)))
        st = oracle.State(g["r"][off_k:off_k + n], g["u"][off_k:off_k + n], g["rho"][off_k:off_k + n],
                          g["type"][off_k:off_k + n])
        ref = oracle.scene(case)
        assert np.array_equal(st.r, ref.r)  # the batch builds the same lattice as the oracle
        st = ref
        sel = _sample(n, 500, 3 + k)
        o = oracle.derivatives_subset(case, st, sel)
        assert normwise(acc[off_k + sel], o[1]) <= MIXED_TOL
        assert normwise(drho[off_k + sel], o[0]) <= MIXED_TOL
    sim.step(0.0, 3)
    dts = sim.last_dt()
    assert len(dts) == 64 and np.all(dts > 0)
    # instances with different alpha and dp take different steps
    assert len(np.unique(np.round(dts, 12))) > 10


def test_fp64_small_dambreak_500_steps_track_the_oracle():
    # The small dam break (7,500 fluid particles) for the 500 adaptive steps of
    # its configuration, FP64 form against the oracle: every dt, the Eq. 33
    # pressures inside the column every 50 steps, and the final state.
    c = wl.small_dambreak()
    case = oracle_case(c)
    st = oracle.scene(case)
    oracle.set_threads(os.cpu_count() or 1)
    sim = sph.Simulation(c, precision=sph.FP64, use_graph=0)
    pts = np.array(c.pressure_xyz)
    floor = 1e-3 * 1000.0 * 9.81 * c.column[2]
    for k in range(500):
        dt_o = oracle.step(case, st)
        sim.step(0.0, 1)
        assert abs(sim.last_dt()[0] - dt_o) <= 1e-8 * dt_o, k
        if k % 50 == 49:
            pg, po = sim.probe_pressure(pts), oracle.probe_pressure(case, st, pts)
            assert np.max(np.abs(pg - po) / np.maximum(np.abs(po), floor)) <= 1e-4, k
    g = sim.get_state()
    assert g["step"] == 500
    assert np.max(np.abs(g["r"] - st.r)) < 1e-8
    assert np.max(np.abs(g["rho"] - st.rho)) < 1e-5


def test_mixed_wave_height_tracks_fp64_over_one_second():
    # The small dam break advanced 1 s of physical time in both forms; wave
    # heights sampled every 0.05 s agree within 2 % of the column height.
    c = wl.small_dambreak()
    pts = np.array(c.wave_xy)
    runs = {}
    for prec in (sph.FP64, sph.MIXED):
        sim = sph.Simulation(c, precision=prec)
        heights = []
        for _ in range(20):
            t_target = (len(heights) + 1) * 0.05
            while sim.time()[0] < t_target:
                sim.step(0.0, 20)
            heights.append(sim.probe_wave_height(pts))
        runs[prec] = np.array(heights)
        assert sim.get_state()["time"][0] >= 1.0
    err = np.abs(runs[sph.MIXED] - runs[sph.FP64]).max() / c.column[2]
    assert err <= 0.02, err


def _still_column(delta, t_end=1.5):
    c = wl.Case("still_column", (0.4, 0.2, 0.4), (0.4, 0.2, 0.2), None, 0.01, alpha=0.1)
    sim = sph.Simulation(c, precision=sph.MIXED, init=sph.INIT_UNIFORM, delta=delta)
    while sim.time()[0] < t_end:
        sim.step(0.0, 200)
    sim.sync()
    pts = np.array([[0.2, 0.1, z] for z in (0.05, 0.08, 0.11, 0.14)])
    p = sim.probe_pressure(pts)
    hw = sim.probe_wave_height(np.array([[0.2, 0.1]]))[0]
    return p, 1000.0 * 9.81 * (hw - pts[:, 2]), hw


def test_still_column_relaxes_to_hydrostatic_pressure():
    # A column covering the whole floor, started at uniform density rho0, must
    # settle to P = rho0 g d (Eq. 8 with the momentum balance of Eq. 3): after
    # 1.5 s the Eq. 33 pressure away from walls, floor and surface is within
    # 2 % of rho0 g d, d measured from the settled surface.  Viscosity 0.1
    # damps the acoustic oscillation.  The delta term is off: the diffusive
    # term of Eq. 7 does not vanish near a free surface and slowly drains the
    # deep density (reported, not asserted, below).
    p, expect, hw = _still_column(0.0)
    assert np.all(np.abs(p - expect) <= 0.02 * expect), (p, expect, hw)
    p1, e1, _ = _still_column(0.1)
    print("delta = 0.1: pressure / rho0 g d =", np.round(p1 / e1, 4))

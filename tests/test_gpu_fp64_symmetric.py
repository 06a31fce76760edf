"""The FP64 pair pass evaluating each interacting pair once
(params.pair_symmetric) against the FP64 oracle and the ordered FP64 pass.

Bars: derivatives normwise <= 1e-6 against the oracle (the FP64 bar; measured
at rounding level); neighbour counts bit-exact against the oracle (the exact
FP64 distance test gives the same decision from both particles); mu_max
bit-identical to the ordered pass (the same pair arithmetic from either
side); 50 adaptive steps tracking the oracle as the ordered FP64 pass is held
(dt to 1e-9 relative, probe pressures to 1e-4, positions to 1e-9 m).
"""
import numpy as np
import pytest

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, normwise, oracle_case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


CASES = [wl.tiny_case(0.04, obstacle=True), wl.small_dambreak()]


@pytest.mark.parametrize("cell_div", [1, 2, 3])
@pytest.mark.parametrize("c", CASES, ids=lambda c: c.name)
def test_fp64_symmetric_derivatives(c, cell_div):
    case = oracle_case(c, cell_div=cell_div)
    st = jittered(c, seed=51, case=case, out_of_domain=2)
    sym = sph.Simulation(c, precision=sph.FP64, pair_symmetric=1, cell_div=cell_div)
    ref = sph.Simulation(c, precision=sph.FP64, cell_div=cell_div)
    load_state(sym, st)
    load_state(ref, st)
    drho, acc, mu, nn = sym.derivatives()
    rd, ra, rm, rn = ref.derivatives()
    o = oracle.derivatives(case, st)
    e = (normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
    assert max(e) <= FP64_TOL, e
    assert max(normwise(drho, rd), normwise(acc, ra)) <= 1e-12
    assert np.array_equal(nn, o[3])
    assert np.array_equal(mu, rm)


def test_fp64_symmetric_coincident_particles():
    # two distinct fluid particles at one position: the r = 0 guard and the
    # delta term's limit, evaluated once and handed to the partner
    c = wl.tiny_case(0.04)
    case = oracle_case(c)
    st = oracle.scene(case)
    f = np.flatnonzero(st.type == oracle.FLUID)
    r = st.r.copy()
    r[f[10]] = r[f[11]]
    rho = st.rho.copy()
    rho[f[10]] += 3.0
    st = oracle.State(r, st.u, rho, st.type)
    sim = sph.Simulation(c, precision=sph.FP64, pair_symmetric=1)
    load_state(sim, st)
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives(case, st)
    assert max(normwise(drho, o[0]), normwise(acc, o[1])) <= FP64_TOL
    assert np.array_equal(nn, o[3])


def test_fp64_symmetric_steps_track_the_oracle():
    c = wl.small_dambreak()
    case = oracle_case(c)
    st = oracle.scene(case)
    sim = sph.Simulation(c, precision=sph.FP64, pair_symmetric=1, use_graph=0)
    pts = np.array(c.pressure_xyz)
    floor = 1e-3 * 1000.0 * 9.81 * c.column[2]
    worst = 0.0
    for _ in range(50):
        dt_o = oracle.step(case, st)
        sim.step(dt=0.0, nsteps=1)
        assert abs(sim.last_dt()[0] - dt_o) <= 1e-9 * dt_o
        pg = sim.probe_pressure(pts)
        po = oracle.probe_pressure(case, st, pts)
        worst = max(worst, float(np.max(np.abs(pg - po) / np.maximum(np.abs(po), floor))))
    assert worst <= 1e-4, worst
    assert np.max(np.abs(sim.get_state()["r"] - st.r)) < 1e-9
    assert sim.launches_per_step() == 10  # the ordered FP64 step's 9 and the finishing kernel


def test_fp64_symmetric_batch_derivatives():
    cases = wl.alpha_sweep(64, seed=2306)[8:11]
    sim = sph.Simulation(cases, precision=sph.FP64, batch=True, pair_symmetric=1)
    off, sl = 0, []
    for k in range(sim.n_inst):
        n = int(sim.counts(k)[3])
        sl.append(slice(off, off + n))
        off += n
    sts = [jittered(c, seed=70 + i) for i, c in enumerate(cases)]
    r = np.vstack([s.r for s in sts]); u = np.vstack([s.u for s in sts]); rho = np.concatenate([s.rho for s in sts])
    sim.set_state(r, u, rho)
    drho, acc, mu, nn = sim.derivatives()
    for i, c in enumerate(cases):
        o = oracle.derivatives(oracle_case(c), sts[i])
        e = (normwise(drho[sl[i]], o[0]), normwise(acc[sl[i]], o[1]), normwise(mu[sl[i]], o[2]))
        assert max(e) <= FP64_TOL, (i, e)
        assert np.array_equal(nn[sl[i]], o[3])


def test_fp64_symmetric_parameters_are_checked():
    c = wl.tiny_case(0.04)
    for kw in ({"precision": sph.MIXED}, {"delta_mode": sph.DELTA_FULL_SUPPORT}):
        args = dict(precision=sph.FP64, pair_symmetric=1)
        args.update(kw)
        with pytest.raises(sph.SphError):
            sph.Simulation(c, **args)

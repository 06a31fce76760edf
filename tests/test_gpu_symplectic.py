"""The symplectic predictor-corrector on the GPU against the oracle's.

FP64 form: 30 adaptive steps of the small dam break from a jittered state
track the oracle step by step (dt to 1e-9 relative, positions to 1e-9 m at the
end, densities and velocities to rounding growth).  Mixed form: 10 steps,
positions within 1e-8 m and densities within 1e-3 kg/m^3.  Graph replay equals
eager launches; the phase accounting shows two pair passes per step.
"""
import numpy as np
import pytest

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, oracle_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _pair(c, prec, seed):
    case = oracle_case(c, integrator=oracle.SYMPLECTIC)
    st = jittered(c, seed=seed, case=case, out_of_domain=2)
    sim = sph.Simulation(c, precision=prec, integrator=sph.SYMPLECTIC, use_graph=0)
    load_state(sim, st)
    return case, st, sim


def test_fp64_symplectic_steps_track_the_oracle():
    c = wl.small_dambreak()
    case, st, sim = _pair(c, sph.FP64, 41)
    for _ in range(30):
        dt_o = oracle.step(case, st)
        sim.step(0.0, 1)
        assert abs(sim.last_dt()[0] - dt_o) <= 1e-9 * dt_o
    g = sim.get_state()
    assert np.max(np.abs(g["r"] - st.r)) < 1e-9
    assert np.max(np.abs(g["u"] - st.u)) < 1e-7
    assert np.max(np.abs(g["rho"] - st.rho)) < 1e-6
    # the level-n state of the last step is the previous level
    assert np.max(np.abs(g["rhoprev"] - st.rhoprev)) < 1e-6
    assert g["step"] == st.step


def test_mixed_symplectic_steps_track_the_oracle():
    c = wl.small_dambreak()
    case, st, sim = _pair(c, sph.MIXED, 43)
    for _ in range(10):
        dt_o = oracle.step(case, st)
        sim.step(0.0, 1)
        assert abs(sim.last_dt()[0] - dt_o) <= 2e-4 * dt_o
    g = sim.get_state()
    assert np.max(np.abs(g["r"] - st.r)) < 1e-8
    assert np.max(np.abs(g["rho"] - st.rho)) < 1e-3


def test_symplectic_graph_replay_equals_eager_and_counts_two_pair_passes():
    c = wl.tiny_case(0.04, obstacle=True)
    a = sph.Simulation(c, precision=sph.MIXED, integrator=sph.SYMPLECTIC, use_graph=1, graph_steps=4)
    b = sph.Simulation(c, precision=sph.MIXED, integrator=sph.SYMPLECTIC, use_graph=0)
    a.step(0.0, 9)
    b.step(0.0, 9)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["r"], sb["r"]) and np.array_equal(sa["u"], sb["u"])
    b.set_profiling(True)
    b.step(0.0, 3)
    ph = b.phase_times()
    b.set_profiling(False)
    assert ph["pair"][1] == 6 and ph["dt"][1] == 3 and ph["integrate"][1] == 6 and ph["reorder"][1] == 6
    assert b.launches_per_step() == 16

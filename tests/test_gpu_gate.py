"""The moving gate (Section 3.2: the Case 2 column is held by a gate lifted at
a constant speed) on the GPU against the oracle.

Gate particles are boundary particles with a prescribed velocity: the scene
matches the oracle's, the pair pass sees their velocity (derivatives within the
usual bars on a jittered state), and adaptive steps of both integrators track
the oracle step by step while the gate rises and the water runs out under it.
"""
import numpy as np
import pytest

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, normwise, oracle_case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
MIXED_TOL = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
def test_gate_scene_matches_oracle(prec):
    c = wl.small_gate_dambreak()
    sim = sph.Simulation(c, precision=prec)
    st = oracle.scene(oracle_case(c))
    g = sim.get_state()
    assert np.array_equal(g["r"], st.r) and np.array_equal(g["type"], st.type)
    gate = st.type == oracle.GATE
    assert gate.sum() == 2 * 25 * 25
    assert np.array_equal(g["u"][gate], st.u[gate]) and np.all(st.u[gate][:, 2] == wl.GATE_SPEED)
    assert tuple(sim.counts()[:3]) == c.lattice_counts()


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
def test_gate_derivatives(prec):
    c = wl.small_gate_dambreak()
    case = oracle_case(c)
    st = jittered(c, seed=19, case=case, out_of_domain=2)
    sim = sph.Simulation(c, precision=prec)
    load_state(sim, st)
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives(case, st)
    tol = FP64_TOL if prec == sph.FP64 else MIXED_TOL
    e = (normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
    assert max(e) <= tol, e
    gate = st.type == oracle.GATE
    # the gate particles next to the water see its motion relative to them
    assert np.abs(o[0][gate]).max() > 0
    assert normwise(drho[gate], o[0][gate]) <= tol


@pytest.mark.parametrize("integ", [sph.VERLET, sph.SYMPLECTIC])
def test_fp64_gate_steps_track_the_oracle(integ):
    c = wl.small_gate_dambreak()
    case = oracle_case(c, integrator=integ)
    st = oracle.scene(case)
    sim = sph.Simulation(c, precision=sph.FP64, integrator=integ, use_graph=0)
    for _ in range(25):
        dt_o = oracle.step(case, st)
        sim.step(0.0, 1)
        assert abs(sim.last_dt()[0] - dt_o) <= 1e-9 * dt_o
    g = sim.get_state()
    assert np.max(np.abs(g["r"] - st.r)) < 1e-9
    assert np.max(np.abs(g["rho"] - st.rho)) < 1e-6
    gate = st.type == oracle.GATE
    t = g["time"][0]
    r0 = oracle.scene(case).r[gate]
    assert np.max(np.abs(g["r"][gate] - (r0 + np.array(c.gate_velocity) * t))) < 1e-12


def test_mixed_gate_steps_track_the_oracle():
    c = wl.small_gate_dambreak()
    case = oracle_case(c)
    st = oracle.scene(case)
    sim = sph.Simulation(c, precision=sph.MIXED, use_graph=0)
    for _ in range(15):
        dt_o = oracle.step(case, st)
        sim.step(0.0, 1)
        assert abs(sim.last_dt()[0] - dt_o) <= 2e-4 * dt_o
    g = sim.get_state()
    assert np.max(np.abs(g["r"] - st.r)) < 1e-8
    assert np.max(np.abs(g["rho"] - st.rho)) < 1e-3

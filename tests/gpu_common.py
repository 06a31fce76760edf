"""Shared helpers of the GPU parity tests."""
import numpy as np

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl


def oracle_case(c: wl.Case, **kw):
    return oracle.make_case(c.tank, c.column, c.obstacle, dp=c.dp, h=c.h, c0=c.c0, rho0=c.rho0, alpha=c.alpha,
                            gate=c.gate, gate_velocity=c.gate_velocity, **kw)


def normwise(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def jittered(c: wl.Case, seed: int, case=None, out_of_domain: int = 0):
    """Oracle scene of case c with seeded noise on positions, velocities and
    densities (fluid moves, boundary keeps u = 0); optionally throws a few
    fluid particles outside the grid."""
    case = case or oracle_case(c)
    st = oracle.scene(case)
    f = st.type == oracle.FLUID
    r, u, rho = wl.perturb(st.r, st.u, st.rho, f, seed, pos_sigma=0.15 * c.dp, vel_sigma=0.3, rho_sigma=2.0)
    if out_of_domain:
        idx = np.flatnonzero(f)[:out_of_domain]
        r[idx, 2] = c.tank[2] + 50.0 * c.h
    return oracle.State(r, u, rho, st.type)


def load_state(sim: sph.Simulation, st: oracle.State):
    sim.set_state(st.r, st.u, st.rho, st.uprev, st.rhoprev, st.step)

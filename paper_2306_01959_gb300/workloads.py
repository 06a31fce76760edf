"""Synthetic dam-break workloads and seeded input generators.

This module holds no arithmetic of the method: only case geometry, constants and
seeded random numbers.  Both the CUDA path (through the C ABI) and the CPU
oracle are fed from here, so that neither side ever produces the other's inputs.

The cases take the shapes of the paper's two 3D dam breaks (a tank with a water
column against one end wall and, in the first, a box obstacle on the floor;
Sections 3.1 and 3.2).  The experimental data those cases were compared with is
not available, so every input is synthetic: lattice particles at rest with a
hydrostatic density, the flow developing from the dam break itself.

Parameters common to all cases: rho0 = 1000 kg/m^3, g = 9.81 m/s^2, gamma = 7,
delta = 0.1, Cr = 0.2, Ns = 40 (Section 2.2 and Section 3), h = 1.2 sqrt(3) dp,
c0 = 10 sqrt(g Hc) with Hc the column height, alpha = 0.01 unless swept.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

G = 9.81
RHO0 = 1000.0
H_FACTOR = 1.2 * math.sqrt(3.0)


@dataclasses.dataclass
class Case:
    """One dam-break instance: geometry [m] and physical parameters."""

    name: str
    tank: Tuple[float, float, float]
    column: Tuple[float, float, float]
    obstacle: Optional[Tuple[float, float, float, float, float, float]]
    dp: float
    alpha: float = 0.01
    h: float = 0.0
    c0: float = 0.0
    rho0: float = RHO0
    steps: int = 500
    sim_time: float = 0.0
    wave_xy: Tuple[Tuple[float, float], ...] = ()
    pressure_xyz: Tuple[Tuple[float, float, float], ...] = ()
    gate: Optional[Tuple[float, float, float, float, float, float]] = None
    gate_velocity: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    def __post_init__(self):
        if self.h == 0.0:
            self.h = H_FACTOR * self.dp
        if self.c0 == 0.0:
            self.c0 = 10.0 * math.sqrt(G * self.column[2])

    def lattice_counts(self, layers: int = 2) -> Tuple[int, int, int]:
        """Fluid, wall+floor (+gate) and obstacle particle counts of the lattice layout."""
        nint = lambda v: int(math.floor(v / self.dp + 0.5))
        nf = nint(self.column[0]) * nint(self.column[1]) * nint(self.column[2])
        tx, ty, tz = nint(self.tank[0]), nint(self.tank[1]), nint(self.tank[2])
        nw = (tx + 2 * layers) * (ty + 2 * layers) * (tz + layers) - tx * ty * tz
        no = 0
        if self.obstacle is not None:
            no = nint(self.obstacle[3]) * nint(self.obstacle[4]) * nint(self.obstacle[5])
        if self.gate is not None:
            nw += nint(self.gate[3]) * nint(self.gate[4]) * nint(self.gate[5])
        return nf, nw, no


def small_dambreak() -> Case:
    """1.0 x 0.5 x 0.5 m tank, 0.4 x 0.5 x 0.3 m column, dp = 0.02 m (7,500 fluid)."""
    return Case("dambreak_small_dp0.02", (1.0, 0.5, 0.5), (0.4, 0.5, 0.3), None, 0.02, steps=500,
                wave_xy=((0.2, 0.25), (0.5, 0.25), (0.8, 0.25)),
                pressure_xyz=((0.1, 0.25, 0.05), (0.2, 0.25, 0.1), (0.3, 0.25, 0.15),
                              (0.05, 0.1, 0.03), (0.35, 0.4, 0.2), (0.2, 0.25, 0.25)))


def _obstacle_case(name: str, dp: float, steps: int) -> Case:
    # Box 0.16 x 0.4 x 0.16 m on the floor, front face 2.4 m from the column's
    # end wall, centred in y.  Eight pressure points: a 2 x 4 grid on the front
    # face; four wave-height probes along the tank centre line.
    py = [0.3 + 0.4 * (k + 0.5) / 4 for k in range(4)]
    pz = [0.16 * (k + 0.5) / 2 for k in range(2)]
    return Case(name, (3.2, 1.0, 1.0), (1.2, 1.0, 0.55), (2.4, 0.3, 0.0, 0.16, 0.4, 0.16), dp,
                steps=steps, sim_time=1.0,
                wave_xy=((0.5, 0.5), (1.5, 0.5), (2.0, 0.5), (2.9, 0.5)),
                pressure_xyz=tuple((2.4, y, z) for z in pz for y in py))


def obstacle_dambreak() -> Case:
    """3.2 x 1.0 x 1.0 m tank, 1.2 x 1.0 x 0.55 m column, box obstacle, dp = 0.01 m."""
    return _obstacle_case("dambreak_obstacle_dp0.01", 0.01, steps=500)


def obstacle_dambreak_fine() -> Case:
    """The obstacle case at dp = 0.005 m (about 5.3 M fluid particles)."""
    return _obstacle_case("dambreak_obstacle_dp0.005", 0.005, steps=100)


def wall_impact() -> Case:
    """1.6 x 0.6 x 0.6 m tank, 0.6 x 0.6 x 0.3 m column, dp = 0.0025 m, far-wall pressure points."""
    return Case("wall_impact_dp0.0025", (1.6, 0.6, 0.6), (0.6, 0.6, 0.3), None, 0.0025, steps=100,
                sim_time=1.0, wave_xy=((0.3, 0.3), (1.2, 0.3)),
                pressure_xyz=tuple((1.6, 0.3, z) for z in (0.003, 0.015, 0.03, 0.08)))


def alpha_sweep(n: int = 64, seed: int = 2306) -> List[Case]:
    """Batched alpha sweep: the small-case tank with column height U[0.2, 0.4] m,
    column length U[0.3, 0.5] m, dp U[0.01, 0.02] m and alpha log-uniform in
    [1e-3, 0.1], drawn from numpy's PCG64 with the given seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        hc = float(rng.uniform(0.2, 0.4))
        lc = float(rng.uniform(0.3, 0.5))
        dp = float(rng.uniform(0.01, 0.02))
        alpha = float(10.0 ** rng.uniform(-3.0, -1.0))
        out.append(Case(f"sweep{k:02d}", (1.0, 0.5, 0.5), (lc, 0.5, hc), None, dp, alpha=alpha, steps=1000,
                        wave_xy=((0.2, 0.25), (0.8, 0.25)), pressure_xyz=((0.05, 0.25, 0.03),)))
    return out


GATE_SPEED = 1.25  # m/s, vertical opening speed of the Case 2 gate (Section 3.2)


def gate_dambreak(dp: float = 0.005) -> Case:
    """A dam break released by a lifting gate, shaped like the paper's Case 2
    (Section 3.2): tank 2.60 x 1.20 x 0.30 m, water column 0.1 m high, gate
    0.025 m thick and 0.30 m high opened upward at 1.25 m/s from t = 0, block
    0.155 x 0.30 x 0.20 m downstream.  The layout figure of that case is not in
    the text; the positions taken here (column 0.5 m long over the full width,
    the gate across the full width at its end, the block's front face 1.0 m
    further, y-centred) are this workload's own."""
    lc = 0.5
    return Case(f"gate_dambreak_dp{dp}", (2.60, 1.20, 0.30), (lc, 1.20, 0.10),
                (lc + 1.0, 0.45, 0.0, 0.155, 0.30, 0.20), dp, steps=200, sim_time=1.0,
                wave_xy=((0.25, 0.6), (1.0, 0.6), (1.45, 0.6)),
                pressure_xyz=((lc + 1.0, 0.6, 0.02), (lc + 1.0, 0.6, 0.06)),
                gate=(lc, 0.0, 0.0, 0.025, 1.20, 0.30), gate_velocity=(0.0, 0.0, GATE_SPEED))


def small_gate_dambreak() -> Case:
    """The small dam break held by a 2-particle-thick gate at the column's end,
    lifted at 1.25 m/s."""
    c = small_dambreak()
    return dataclasses.replace(c, name="gate_small_dp0.02", gate=(c.column[0], 0.0, 0.0, 2 * c.dp, c.tank[1], c.tank[2]),
                               gate_velocity=(0.0, 0.0, GATE_SPEED))


def paper_parameters(c: Case) -> Case:
    """The same case with the paper's own numerical parameters: 2h = 3 l0
    (h = 1.5 dp) and c0 = 20 sqrt(g H_W), H_W the column height (Section 3)."""
    return dataclasses.replace(c, name=c.name + "_paper", h=1.5 * c.dp, c0=20.0 * math.sqrt(G * c.column[2]))


def paper_case1() -> Case:
    """The obstacle dam break at the paper's Case 1 resolution l0 = 0.0075 m
    (about 1.55 M fluid particles, the size of its Table 1 run) with the paper's
    h and c0."""
    return paper_parameters(_obstacle_case("dambreak_obstacle_dp0.0075", 0.0075, steps=200))


MPS_CASE1_DT = 3.0e-4  # s, the fixed MPS time step of Table 1 (l0 = 0.0075 m)


def mps_case1() -> Case:
    """The paper's Case 1 tank shape for the MPS step (Section 3.1, Table 1):
    tank 3.22 x 1.0 x 1.0 m, column 1.2 x 1.0 x 0.55 m, l0 = 0.0075 m (1.55 M
    fluid and, with three wall layers, 0.64 M wall and dummy particles); the
    box obstacle is left out (the MPS step here has fixed walls only)."""
    return Case("mps_dambreak_l0.0075", (3.22, 1.0, 1.0), (1.2, 1.0, 0.55), None, 0.0075, steps=20)


def by_name(name: str) -> Case:
    table = {c().name: c for c in (small_dambreak, obstacle_dambreak, obstacle_dambreak_fine, wall_impact,
                                    paper_case1, gate_dambreak, small_gate_dambreak)}
    return table[name]()


def tiny_case(dp: float = 0.05, obstacle: bool = False) -> Case:
    """A coarse tank for quick checks (a few thousand particles)."""
    ob = (0.6, 0.1, 0.0, 0.1, 0.2, 0.1) if obstacle else None
    return Case(f"tiny_dp{dp}", (1.0, 0.4, 0.4), (0.3, 0.4, 0.2), ob, dp, steps=50,
                wave_xy=((0.1, 0.2), (0.7, 0.2)), pressure_xyz=((0.1, 0.2, 0.05), (0.2, 0.2, 0.1)))


def perturb(r: np.ndarray, u: np.ndarray, rho: np.ndarray, fluid: np.ndarray, seed: int, *, pos_sigma: float,
            vel_sigma: float, rho_sigma: float, rho0: float = RHO0):
    """Seeded random perturbation of a lattice state (fluid particles only move;
    boundary particles keep u = 0 but get density noise).  Returns new arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = r.shape[0]
    dr = rng.normal(0.0, pos_sigma, size=(n, 3))
    du = rng.normal(0.0, vel_sigma, size=(n, 3))
    drho = rng.normal(0.0, rho_sigma, size=n)
    f = fluid.astype(bool)
    r2 = r.copy()
    r2[f] += dr[f]
    u2 = u.copy()
    u2[f] += du[f]
    rho2 = rho + drho
    return r2, u2, rho2


def random_points(lo, hi, n: int, seed: int) -> np.ndarray:
    """n uniform points in the box [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return lo + (hi - lo) * rng.random((n, 3))

"""Further parity of the CUDA path with the FP64 CPU oracle.

- the delta term of Eq. 7 dropped next to boundaries (SPH_DELTA_FULL_SUPPORT),
  in both forms;
- the mixed form's cell ids and per-cell particle sets against the oracle's
  counting sort, and its neighbour counts;
- two distinct particles at one position (the r = 0 limit of the delta term
  and of the distance guards);
- a batch of instances stepped with adaptive, per-instance dt against the
  oracle run of every instance, and mu_max of a batch pass;
- a regression bar for the mixed form near its measured error (the tolerance
  of the method stays 2e-4; the compensated sums reach a few 1e-7);
- a still column with delta = 0.1 over full supports holding the hydrostatic
  pressure on the GPU as on the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, normwise, oracle_case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
MIXED_TOL = 2e-4
MIXED_REGRESSION = 5e-6  # measured 3-4e-7 with compensated sums


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


CASES = [wl.tiny_case(0.04, obstacle=True), wl.small_dambreak()]


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
@pytest.mark.parametrize("c", CASES, ids=lambda c: c.name)
def test_derivatives_delta_full_support(c, prec):
    case = oracle_case(c, delta_mode=oracle.DELTA_FULL_SUPPORT)
    st = jittered(c, seed=41, case=case, out_of_domain=2)
    sim = sph.Simulation(c, precision=prec, delta_mode=sph.DELTA_FULL_SUPPORT)
    load_state(sim, st)
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives(case, st)
    e = (normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
    assert max(e) <= (FP64_TOL if prec == sph.FP64 else MIXED_REGRESSION), e
    # the mode changes the density rates of exactly the fluid particles that
    # touch a boundary particle: compare with the default mode's rates
    o_all = oracle.derivatives(oracle_case(c), st)
    changed = np.abs(o_all[0] - o[0]) > 0
    assert changed.sum() > 50
    assert np.all(st.type[changed] == oracle.FLUID)
    if prec == sph.FP64:
        assert np.array_equal(nn, o[3])
        assert np.max(np.abs(drho - o[0])) <= 1e-9 * np.abs(o[0]).max()


@pytest.mark.parametrize("c", CASES, ids=lambda c: c.name)
def test_mixed_derivatives_regression_bar(c):
    case = oracle_case(c, cell_div=1)
    st = jittered(c, seed=5, case=case, out_of_domain=2)
    sim = sph.Simulation(c, precision=sph.MIXED)
    load_state(sim, st)
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives(case, st)
    e = (normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
    assert max(e) <= MIXED_REGRESSION, e


@pytest.mark.parametrize("c", CASES, ids=lambda c: c.name)
def test_mixed_cells_and_cell_sets_match_oracle(c):
    # The mixed form bins with a multiplication by 1/cs (the FP64 form divides);
    # the two differ only for a coordinate within one rounding of a cell face,
    # which the seeded positions avoid (checked below).  Within a cell the mixed
    # form orders by x, so the cells are compared as sets.
    case = oracle_case(c, cell_div=1)
    st = jittered(c, seed=13, case=case, out_of_domain=4)
    lo, size, dims = oracle.grid_info(case)
    scaled = (st.r - lo) / size
    assert np.min(np.abs(scaled - np.round(scaled))) > 1e-9
    sim = sph.Simulation(c, precision=sph.MIXED)
    load_state(sim, st)
    cell, srt, start = sim.cells()
    o_cell, o_order, o_start = oracle.cells(case, st.r)
    assert np.array_equal(cell, o_cell)
    assert np.array_equal(start, o_start[:-1])
    n_in = int(o_start[-2])
    assert len(srt) == n_in
    by_cell_then_id = srt[np.lexsort((srt, cell[srt]))]
    assert np.array_equal(by_cell_then_id, o_order[:n_in])
    # within each cell the mixed order is by x
    xs = st.r[srt, 0]
    same = cell[srt][1:] == cell[srt][:-1]
    assert np.all(xs[1:][same] >= xs[:-1][same])
    # neighbour counts: FP32 offsets can move a pair across |r| = 2h only within
    # one FP32 rounding of the support radius
    _, _, _, nn = sim.derivatives()
    o_nn = oracle.neighbour_counts(case, st.r)
    diff = np.flatnonzero(nn != o_nn)
    assert len(diff) <= 4 and np.all(np.abs(nn[diff] - o_nn[diff]) <= 1), (len(diff), nn[diff], o_nn[diff])


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
def test_coincident_distinct_particles(prec):
    # Pairs of distinct fluid particles at one position: the delta term takes
    # its r -> 0 limit (-F(0)), every other term vanishes for the pair.
    c = wl.small_dambreak()
    case = oracle_case(c)
    st = jittered(c, seed=23, case=case)
    f = np.flatnonzero(st.type == oracle.FLUID)
    rng = np.random.Generator(np.random.PCG64(23))
    a = rng.choice(f, size=40, replace=False)
    r = st.r.copy()
    r[a[:20]] = r[a[20:]]
    st = oracle.State(r, st.u, st.rho, st.type)
    sim = sph.Simulation(c, precision=prec)
    load_state(sim, st)
    drho, acc, mu, nn = sim.derivatives()
    o = oracle.derivatives(case, st)
    tol = FP64_TOL if prec == sph.FP64 else MIXED_REGRESSION
    e = (normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
    assert max(e) <= tol, e
    assert normwise(drho[a], o[0][a]) <= tol * 10
    if prec == sph.FP64:
        assert np.array_equal(nn, o[3])
    assert np.all(np.isfinite(drho)) and np.all(np.isfinite(acc))


def _instance_slices(sim):
    off = 0
    out = []
    for k in range(sim.n_inst):
        n = int(sim.counts(k)[3])
        out.append(slice(off, off + n))
        off += n
    return out


def test_batch_steps_track_the_oracle_per_instance():
    # Four instances of the alpha sweep (different dp, column, alpha) in one
    # batch, FP64 form, 12 adaptive steps: every instance's dt each step and its
    # final state against the oracle run of that instance alone.
    cases = wl.alpha_sweep(64, seed=2306)[:4]
    sim = sph.Simulation(cases, precision=sph.FP64, batch=True)
    sl = _instance_slices(sim)
    ocases = [oracle_case(c) for c in cases]
    sts = [oracle.scene(oc) for oc in ocases]
    for k in range(12):
        sim.step(0.0, 1)
        dts = sim.last_dt()
        for i, (oc, st) in enumerate(zip(ocases, sts)):
            dt_o = oracle.step(oc, st)
            assert abs(dts[i] - dt_o) <= 1e-9 * dt_o, (k, i, dts[i], dt_o)
    assert len(np.unique(np.round(dts, 14))) == 4
    g = sim.get_state()
    for i, st in enumerate(sts):
        assert np.max(np.abs(g["r"][sl[i]] - st.r)) < 1e-10
        assert np.max(np.abs(g["rho"][sl[i]] - st.rho)) < 1e-7
        assert np.max(np.abs(g["u"][sl[i]] - st.u)) < 1e-8


@pytest.mark.parametrize("prec", [sph.FP64, sph.MIXED])
def test_batch_derivatives_with_mu_max(prec):
    cases = wl.alpha_sweep(64, seed=2306)[4:8]
    sim = sph.Simulation(cases, precision=prec, batch=True)
    sl = _instance_slices(sim)
    sts = []
    for i, c in enumerate(cases):
        sts.append(jittered(c, seed=60 + i))
    r = np.vstack([s.r for s in sts]); u = np.vstack([s.u for s in sts]); rho = np.concatenate([s.rho for s in sts])
    sim.set_state(r, u, rho)
    drho, acc, mu, nn = sim.derivatives()
    tol = FP64_TOL if prec == sph.FP64 else MIXED_REGRESSION
    for i, c in enumerate(cases):
        o = oracle.derivatives(oracle_case(c), sts[i])
        e = (normwise(drho[sl[i]], o[0]), normwise(acc[sl[i]], o[1]), normwise(mu[sl[i]], o[2]))
        assert max(e) <= tol, (i, e)
        assert np.max(o[2]) > 0.0
        if prec == sph.FP64:
            assert np.array_equal(nn[sl[i]], o[3])


def test_gpu_still_column_with_delta_over_full_supports():
    # delta = 0.1 over full supports, symplectic steps: the still column holds
    # the hydrostatic pressure on the GPU (mixed form), within 2 % at points from
    # 2h above the floor to 4h below the surface, the surface being where the
    # fitted pressure profile vanishes, within dp/2 of the particle surface.
    # At dp = 0.01 m the viscosity of Eq. 32 damps the column's acoustic
    # oscillation slowly, so the pressures are averaged over 1.0-1.5 s.
    dp = 0.01
    c = wl.Case("still_column", (0.3, 0.2, 0.5), (0.3, 0.2, 0.4), None, dp, alpha=0.1)
    sim = sph.Simulation(c, precision=sph.MIXED, init=sph.INIT_UNIFORM, delta_mode=sph.DELTA_FULL_SUPPORT,
                         integrator=sph.SYMPLECTIC)
    while sim.time()[0] < 1.0:
        sim.step(0.0, 100)
    sim.sync()
    g = sim.get_state()
    zf = g["r"][g["type"] == 0, 2]
    zs = zf[zf > zf.max() - 0.5 * dp].mean() + 0.5 * dp
    pts = np.array([[0.15, 0.1, z] for z in np.arange(2 * c.h, zs - 4 * c.h, 2 * dp)])
    samples = []
    while sim.time()[0] < 1.5:
        sim.step(0.0, 20)
        samples.append(sim.probe_pressure(pts))
    p = np.mean(samples, axis=0)
    a, b = np.polyfit(pts[:, 2], p, 1)
    z0 = -b / a
    ratio = p / (1000.0 * 9.81 * (z0 - pts[:, 2]))
    assert np.all(np.abs(ratio - 1.0) <= 0.02), ratio
    assert abs(a / (-1000.0 * 9.81) - 1.0) <= 0.02
    assert abs(z0 - zs) <= 0.5 * dp

"""The persistent time loop: one cooperative launch per sph_step call.

Its phases are the per-phase kernels' bodies separated by grid barriers, so a
batch advanced persistently must equal the same batch advanced by per-phase
launches bit for bit (both run the pair pass in its default shape with
compensated sums).  Every barrier wait is bounded: with a spin limit of one
poll the waits run out, the launch ends, sph_sync reports SPH_ETIMEOUT, and the
context stays usable.
"""
import numpy as np
import pytest

from paper_2306_01959_gb300 import sph, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


SHAPE = dict(pair_warps=8, pair_ctas_per_sm=2, pair_group=4, compensated=1)


@pytest.mark.parametrize("delta_mode", [sph.DELTA_ALL_FLUID, sph.DELTA_FULL_SUPPORT])
def test_persistent_batch_equals_per_phase_launches(delta_mode):
    cases = wl.alpha_sweep(64, seed=2306)[:6]
    a = sph.Simulation(cases, precision=sph.MIXED, batch=True, persistent=1, delta_mode=delta_mode, **SHAPE)
    b = sph.Simulation(cases, precision=sph.MIXED, batch=True, use_graph=1, graph_steps=5, delta_mode=delta_mode,
                       **SHAPE)
    for chunk in (1, 4, 40):  # crosses the first-order steps at 0 and 40
        a.step(0.0, chunk)
        b.step(0.0, chunk)
    a.sync()
    b.sync()
    ga, gb = a.get_state(), b.get_state()
    assert ga["step"] == gb["step"] == 45
    for k in ("r", "u", "rho", "uprev", "rhoprev", "time"):
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(a.last_dt(), b.last_dt())
    ca, cb = a.cells(), b.cells()
    for x, y in zip(ca, cb):
        assert np.array_equal(x, y)


def test_persistent_single_tank_with_fixed_dt():
    c = wl.small_dambreak()
    a = sph.Simulation(c, precision=sph.MIXED, persistent=1, **SHAPE)
    b = sph.Simulation(c, precision=sph.MIXED, use_graph=0, **SHAPE)
    a.step(2e-4, 30)
    b.step(2e-4, 30)
    ga, gb = a.get_state(), b.get_state()
    assert np.array_equal(ga["r"], gb["r"]) and np.array_equal(ga["rho"], gb["rho"])
    assert abs(ga["time"][0] - 30 * 2e-4) < 1e-15


def test_persistent_rejects_unsupported_forms():
    c = wl.tiny_case()
    for kw in (dict(precision=sph.FP64), dict(precision=sph.MIXED, integrator=sph.SYMPLECTIC)):
        with pytest.raises(sph.SphError):
            sph.Simulation(c, persistent=1, **kw)


def test_barrier_wait_runs_out_and_reports_timeout():
    # A spin limit of one poll: every CTA but the last to arrive gives up at the
    # first barrier, records the timeout and returns; the last one gives up at
    # the next.  The launch ends, the status reads SPH_ETIMEOUT.
    cases = wl.alpha_sweep(64, seed=2306)[:3]
    sim = sph.Simulation(cases, precision=sph.MIXED, batch=True, persistent=1, spin_limit=1)
    sim.step(0.0, 3)
    with pytest.raises(sph.SphError) as e:
        sim.sync()
    assert e.value.code == sph.SPH_ETIMEOUT
    sim.close()
    # the context is still usable
    ok = sph.Simulation(cases, precision=sph.MIXED, batch=True, persistent=1)
    ok.step(0.0, 3)
    ok.sync()
    assert np.all(ok.last_dt() > 0)

"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point include/sph.h declares.  No compute calls."""
import ctypes
import os
import re

import pytest

from paper_2306_01959_gb300 import build, sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols(header="sph.h", prefix="sph"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sph.load()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ["sph_create", "sph_step", "sph_probe", "sph_batch_create", "sph_get_state", "sph_set_state",
                 "sph_derivatives", "sph_workspace_size", "sph_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    assert set(_declared_symbols()) == set(sph.SIGNATURES), "binding and header disagree"


def test_library_exports_every_mps_symbol(lib):
    from paper_2306_01959_gb300 import mps

    names = _declared_symbols("mps.h", "mps")
    for must in ["mps_create", "mps_step", "mps_pressure", "mps_get_state", "mps_workspace_size"]:
        assert must in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(mps.SIGNATURES), "MPS binding and header disagree"
    p = mps.default_params()
    assert p.size == ctypes.sizeof(mps.Params)
    assert (p.re_factor, p.kappa_c, p.kappa_r, p.beta1, p.varrho1, p.layers) == (2.1, 1e-8, 0.01, 0.98, 0.2, 3)
    n = ctypes.c_size_t()
    t3 = (ctypes.c_double * 3)(0.24, 0.24, 0.4)
    c3 = (ctypes.c_double * 3)(0.24, 0.24, 0.3)
    assert lib.mps_workspace_size(t3, c3, 0.02, ctypes.byref(p), ctypes.byref(n)) == 0 and n.value > 0
    bad = (ctypes.c_double * 3)(0.5, 0.24, 0.3)  # column longer than the tank
    assert lib.mps_workspace_size(t3, bad, 0.02, ctypes.byref(p), ctypes.byref(n)) == sph.SPH_EINVAL


def test_struct_sizes_match_header(lib):
    p = sph.Params()
    lib.sph_params_default(ctypes.byref(p))
    assert p.size == ctypes.sizeof(sph.Params)
    assert (p.gamma, p.g, p.delta, p.cfl, p.ns) == (7.0, 9.81, 0.1, 0.2, 40)


def test_workspace_size_and_validation(lib):
    from paper_2306_01959_gb300 import workloads as wl
    c = wl.small_dambreak()
    p = sph.default_params()
    inst = (sph.Instance * 1)(sph.make_instance(c))
    n = ctypes.c_size_t()
    assert lib.sph_workspace_size(1, inst, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value > (7500 + 11032) * 200
    bad = sph.make_instance(c)
    bad.dp = -1.0
    assert lib.sph_workspace_size(1, (sph.Instance * 1)(bad), ctypes.byref(p), ctypes.byref(n)) == sph.SPH_EINVAL
    bad = sph.make_instance(c)
    bad.column[0] = 5.0  # longer than the tank
    assert lib.sph_workspace_size(1, (sph.Instance * 1)(bad), ctypes.byref(p), ctypes.byref(n)) == sph.SPH_EINVAL
    p2 = sph.default_params(cell_div=7)
    assert lib.sph_workspace_size(1, inst, ctypes.byref(p2), ctypes.byref(n)) == sph.SPH_EINVAL
    assert sph.default_params().integrator == sph.VERLET
    p4 = sph.default_params(integrator=sph.SYMPLECTIC)
    assert lib.sph_workspace_size(1, inst, ctypes.byref(p4), ctypes.byref(n)) == 0
    p4.integrator = 2
    assert lib.sph_workspace_size(1, inst, ctypes.byref(p4), ctypes.byref(n)) == sph.SPH_EINVAL
    p3 = sph.default_params()
    p3.size = 4
    assert lib.sph_workspace_size(1, inst, ctypes.byref(p3), ctypes.byref(n)) == sph.SPH_EINVAL
    ob = sph.make_instance(wl.obstacle_dambreak())
    ob.obstacle[0] = 0.5  # inside the column
    assert lib.sph_workspace_size(1, (sph.Instance * 1)(ob), ctypes.byref(p), ctypes.byref(n)) == sph.SPH_EINVAL


def test_null_handle_calls_are_rejected(lib):
    assert lib.sph_step(None, 0.0, 1) == sph.SPH_EINVAL
    assert lib.sph_sync(None) == sph.SPH_EINVAL
    assert lib.sph_last_error(None) == b"null handle"
    assert lib.sph_num_phases() == 6


def test_neighbour_list_and_each_pair_once_options(lib):
    # Host logic of the two opt-in passes, through sph_workspace_size (no GPU):
    # the combinations each one supports, and the workspace each one adds.
    import math

    from paper_2306_01959_gb300 import workloads as wl
    c = wl.small_dambreak()
    inst = (sph.Instance * 1)(sph.make_instance(c))
    N = 7500 + 11032
    n = ctypes.c_size_t()

    def size(**kw):
        rc = lib.sph_workspace_size(1, inst, ctypes.byref(sph.default_params(**kw)), ctypes.byref(n))
        return rc, n.value

    # neighbour lists: mixed form, Verlet, per-phase launches, cell_div 1
    for kw in ({"precision": sph.FP64}, {"integrator": sph.SYMPLECTIC}, {"persistent": 1}, {"cell_div": 2}):
        args = dict(precision=sph.MIXED, list_skin=0.3)
        args.update(kw)
        assert size(**args)[0] == sph.SPH_EINVAL, kw
    for kw in ({"list_skin": -0.1}, {"list_skin": 5.0}, {"list_skin": 0.3, "list_capacity": -1}):
        assert size(precision=sph.MIXED, **kw)[0] == sph.SPH_EINVAL, kw
    # every entry per particle is 4 bytes; each workspace array starts on 256 bytes
    rc64, s64 = size(precision=sph.MIXED, list_skin=0.3, list_capacity=64)
    rc96, s96 = size(precision=sph.MIXED, list_skin=0.3, list_capacity=96)
    assert rc64 == rc96 == 0 and abs((s96 - s64) - 4 * 32 * N) < 256
    # automatic capacity: the lattice count within 2h + s, plus a third, in multiples of 32
    rc0, s0 = size(precision=sph.MIXED, list_skin=0.3)
    R = (2.0 + 0.3) * c.h / c.dp
    cap = math.ceil(4.0 / 3.0 * math.pi * R ** 3 * 4.0 / 3.0 / 32.0) * 32
    assert rc0 == 0 and abs((s0 - s64) - 4 * (cap - 64) * N) < 256
    # each pair once: FP64 form with the delta term over all fluid pairs; 44 bytes per particle
    assert size(precision=sph.MIXED, pair_symmetric=1)[0] == sph.SPH_EINVAL
    assert size(precision=sph.FP64, pair_symmetric=1, delta_mode=sph.DELTA_FULL_SUPPORT)[0] == sph.SPH_EINVAL
    rcs, ss = size(precision=sph.FP64, pair_symmetric=1)
    rcn, sn = size(precision=sph.FP64)
    assert rcs == rcn == 0 and abs((ss - sn) - 44 * N) < 3 * 256

"""Shared-memory bounds of the mixed pair kernel, checked by the kernel itself.

The library is rebuilt with -DSPH_DEBUG: before every write into its staging
buffers and candidate lists the kernel checks the index, records a failed check
in the device status (reported as SPH_ESTATE) and skips the write.  The cases
that push those indices furthest run on it: neighbourhoods beyond the staging
capacity (a dense clump processed in chunks) at every cell size and group
size, with row windows longer than a candidate list.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np
import oracle
from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, normwise, oracle_case
import test_gpu_parity as P
assert sph.lib_path().endswith("_build_debug/libsph.so")
c = wl.small_dambreak()
for cell_div in (1, 2, 3):
    st = P._clumped(c, 2600, seed=17)
    o = oracle.derivatives(oracle_case(c, cell_div=cell_div), st)
    for group in (1, 2, 4):
        sim = sph.Simulation(c, precision=sph.MIXED, cell_div=cell_div, pair_group=group)
        load_state(sim, st)
        drho, acc, mu, nn = sim.derivatives()
        sim.sync()  # raises SPH_ESTATE if a bounds check failed
        e = max(normwise(drho, o[0]), normwise(acc, o[1]), normwise(mu, o[2]))
        assert e <= 2e-4, (cell_div, group, e)
        sim.step(0.0, 2)
        sim.sync()
        sim.close()
print("bounds: ok")
"""


def test_mixed_pair_kernel_bounds_checked_build():
    from paper_2306_01959_gb300 import build as b

    lib = b.build(debug=True)
    env = dict(os.environ, SPH_LIB=lib)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "bounds: ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]

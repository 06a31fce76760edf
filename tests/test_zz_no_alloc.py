"""The allocation-free time-step entry point against the handle-based one.

sph_cfl_dt_noalloc serves callers that cannot allocate device memory (plug-ins
whose host application's allocator owns the device, real-time loops that must
not risk an allocation's synchronisation, fixed memory budgets); it keeps its
scratch in a fixed device array of the library.  This test feeds it the
derivatives of a state and compares its step with the one sph_step takes on the
same state, twice in a row (the shared scratch must not leak between calls),
then once without a type array over the fluid particles alone.  The device
buffers here are the test's own.
"""
import numpy as np
import pytest

from paper_2306_01959_gb300 import sph, workloads as wl
from gpu_common import jittered, load_state, oracle_case

pytestmark = pytest.mark.gpu


def test_noalloc_dt_matches_sph_step_twice():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    c = wl.small_dambreak()
    st = jittered(c, seed=17, case=oracle_case(c), out_of_domain=3)
    sim = sph.Simulation(c, precision=sph.FP64)
    load_state(sim, st)
    drho, acc, mumax, nneigh = sim.derivatives()
    sim.step(0.0, 1)
    dt_ref = float(sim.last_dt()[0])
    # particle types with the out-of-domain particles excluded
    ty = np.where(nneigh < 0, -1, st.type).astype(np.int32)
    d_acc = torch.tensor(acc, dtype=torch.float64, device="cuda")
    d_mu = torch.tensor(mumax, dtype=torch.float64, device="cuda")
    d_ty = torch.tensor(ty, dtype=torch.int32, device="cuda")
    d_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        d_out.fill_(-1.0)
        sph.cfl_dt_noalloc(d_acc.data_ptr(), d_mu.data_ptr(), d_ty.data_ptr(), len(ty), c.h, c.c0, 0.2,
                           d_out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        dt = float(d_out.item())
        assert abs(dt - dt_ref) <= 1e-12 * dt_ref, (dt, dt_ref)
    # without a type array every particle counts: the fluid particles come
    # first in id order, so the first nf of them give the same step
    nf = int(sim.counts()[0])
    sph.cfl_dt_noalloc(d_acc.data_ptr(), d_mu.data_ptr(), 0, nf, c.h, c.c0, 0.2, d_out.data_ptr(),
                       stream.cuda_stream)
    torch.cuda.synchronize()
    assert abs(float(d_out.item()) - dt_ref) <= 1e-12 * dt_ref
    with pytest.raises(sph.SphError):
        sph.cfl_dt_noalloc(d_acc.data_ptr(), d_mu.data_ptr(), 0, (1 << 24) + 1, c.h, c.c0, 0.2,
                           d_out.data_ptr(), stream.cuda_stream)

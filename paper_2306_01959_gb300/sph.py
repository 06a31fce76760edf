"""Python binding of the C ABI in ``include/sph.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libsph.so``; this module
only converts arguments.  PyTorch provides the device workspace (one uint8
tensor) and the CUDA stream.  Loading fails loudly when the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_EUNSTABLE, SPH_ETIMEOUT, SPH_ESTATE = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
INIT_HYDROSTATIC, INIT_UNIFORM = 0, 1
CSOUND_EOS, CSOUND_CONSTANT = 0, 1
VERLET, SYMPLECTIC = 0, 1
DELTA_ALL_FLUID, DELTA_FULL_SUPPORT = 0, 1
FLUID, WALL, OBSTACLE, GATE = 0, 1, 2, 3
PROBE_PRESSURE, PROBE_WAVE_HEIGHT, PROBE_FORCE = 0, 1, 2

_ERRNAMES = {SPH_EINVAL: "SPH_EINVAL", SPH_ENOMEM: "SPH_ENOMEM", SPH_ECUDA: "SPH_ECUDA",
             SPH_EUNSTABLE: "SPH_EUNSTABLE", SPH_ETIMEOUT: "SPH_ETIMEOUT", SPH_ESTATE: "SPH_ESTATE"}


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("g", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("dt_min", ctypes.c_double),
        ("ns", ctypes.c_int32),
        ("boundary_layers", ctypes.c_int32),
        ("init", ctypes.c_int32),
        ("csound", ctypes.c_int32),
        ("cell_div", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("pair_warps", ctypes.c_int32),
        ("pair_ctas_per_sm", ctypes.c_int32),
        ("compensated", ctypes.c_int32),
        ("pair_group", ctypes.c_int32),
        ("integrator", ctypes.c_int32),
        ("delta_mode", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("spin_limit", ctypes.c_int32),
        ("list_capacity", ctypes.c_int32),
        ("list_skin", ctypes.c_double),
        ("pair_symmetric", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class Instance(ctypes.Structure):
    _fields_ = [
        ("tank", ctypes.c_double * 3),
        ("column", ctypes.c_double * 3),
        ("has_obstacle", ctypes.c_int32),
        ("has_gate", ctypes.c_int32),
        ("obstacle", ctypes.c_double * 6),
        ("dp", ctypes.c_double),
        ("h", ctypes.c_double),
        ("c0", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("gate", ctypes.c_double * 6),
        ("gate_velocity", ctypes.c_double * 3),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p

# Every entry point of include/sph.h with its ctypes signature.
SIGNATURES = {
    "sph_params_default": (None, [ctypes.POINTER(Params)]),
    "sph_workspace_size": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Instance), ctypes.POINTER(Params),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "sph_create": (ctypes.c_int, [ctypes.POINTER(_VP), _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Params), _VP,
                                  ctypes.c_size_t, ctypes.c_size_t]),
    "sph_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int32, ctypes.POINTER(Instance),
                                        ctypes.POINTER(Params), _VP, ctypes.c_size_t, ctypes.c_size_t]),
    "sph_destroy": (None, [_VP]),
    "sph_step": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int32]),
    "sph_sync": (ctypes.c_int, [_VP]),
    "sph_probe": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _D, ctypes.c_int32, _D]),
    "sph_counts": (ctypes.c_int, [_VP, ctypes.c_int32, _I64]),
    "sph_sizes": (ctypes.c_int, [_VP, _I32, _I64, _I64]),
    "sph_get_state": (ctypes.c_int, [_VP, _D, _D, _D, _I32, _D, _D, _I64, _D]),
    "sph_set_state": (ctypes.c_int, [_VP, _D, _D, _D, _D, _D, ctypes.c_int64, _D]),
    "sph_derivatives": (ctypes.c_int, [_VP, _D, _D, _D, _I32]),
    "sph_cells": (ctypes.c_int, [_VP, _I64, _I64, _I64, _I64]),
    "sph_last_dt": (ctypes.c_int, [_VP, _D]),
    "sph_diagnostics": (ctypes.c_int, [_VP, ctypes.c_int32, _D]),
    "sph_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "sph_phase_times": (ctypes.c_int, [_VP, _D, _I64, ctypes.c_int32]),
    "sph_phase_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "sph_num_phases": (ctypes.c_int32, []),
    "sph_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, _I32]),
    "sph_pair_stats": (ctypes.c_int, [_VP, _I64]),
    "sph_tuned_config": (ctypes.c_int, [_VP, _I32]),
    "sph_launches_per_step": (ctypes.c_int32, [_VP]),
    "sph_list_stats": (ctypes.c_int, [_VP, _I64]),
    "sph_last_error": (ctypes.c_char_p, [_VP]),
    "sph_alu_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_size_t, _D]),
    "sph_cfl_dt_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _VP, ctypes.c_size_t]),
}

_lib = None


def lib_path() -> str:
    """The library to load: SPH_LIB if set (e.g. the bounds-checked debug
    build), else the in-tree release build."""
    return os.environ.get("SPH_LIB") or _build.LIB


def load(path: Optional[str] = None):
    """Load libsph.so and bind every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_params(**kw) -> Params:
    p = Params()
    load().sph_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def make_instance(case) -> Instance:
    """Instance from a workloads.Case (or any object with the same fields)."""
    inst = Instance()
    inst.tank[:] = [float(v) for v in case.tank]
    inst.column[:] = [float(v) for v in case.column]
    if case.obstacle is not None:
        inst.has_obstacle = 1
        inst.obstacle[:] = [float(v) for v in case.obstacle]
    inst.dp, inst.h, inst.c0, inst.rho0, inst.alpha = case.dp, case.h, case.c0, case.rho0, case.alpha
    gate = getattr(case, "gate", None)
    if gate is not None:
        inst.has_gate = 1
        inst.gate[:] = [float(v) for v in gate]
        inst.gate_velocity[:] = [float(v) for v in case.gate_velocity]
    return inst


def _d(a):
    return a.ctypes.data_as(_D)


def _opt(a, ptr):
    return ptr(a) if a is not None else None


def cfl_dt_noalloc(acc_ptr, mumax_ptr, type_ptr, n, h, c0, cfl, dt_out_ptr, stream=0):
    """Allocation-free Eq. 15 step from device pointers (see sph_cfl_dt_noalloc)."""
    rc = load().sph_cfl_dt_noalloc(acc_ptr, mumax_ptr, type_ptr, int(n), float(h), float(c0), float(cfl),
                                   dt_out_ptr, int(stream))
    if rc != SPH_OK:
        raise SphError(rc, "sph_cfl_dt_noalloc failed")


def alu_peak(precision, millis=100, stream=0):
    """Measured FMA throughput in flop/s (sph_alu_peak): FP32 for MIXED, FP64 for FP64."""
    out = ctypes.c_double()
    rc = load().sph_alu_peak(int(precision), int(millis), int(stream), ctypes.byref(out))
    if rc != SPH_OK:
        raise SphError(rc, "sph_alu_peak failed")
    return out.value


class Simulation:
    """One handle of the C library: a single tank or a batch of instances."""

    def __init__(self, cases, params: Optional[Params] = None, device="cuda", batch: Optional[bool] = None,
                 **param_kw):
        import torch

        L = load()
        if not isinstance(cases, (list, tuple)):
            cases = [cases]
        self.cases = list(cases)
        self.params = params if params is not None else default_params(**param_kw)
        arr = (Instance * len(self.cases))(*[make_instance(c) for c in self.cases])
        nbytes = ctypes.c_size_t()
        rc = L.sph_workspace_size(len(self.cases), arr, ctypes.byref(self.params), ctypes.byref(nbytes))
        if rc != SPH_OK:
            raise SphError(rc, "invalid instance or parameters")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.workspace.device)
        self._h = _VP()
        single = len(self.cases) == 1 if batch is None else not batch
        # sph_create takes the paper's scalar arguments only; an instance with a
        # gate is created through the instance array
        single = single and not arr[0].has_gate
        if single:
            c = arr[0]
            ob = c.obstacle if c.has_obstacle else None
            rc = L.sph_create(ctypes.byref(self._h), c.tank, c.column, ob, c.dp, c.h, c.c0, c.rho0, c.alpha,
                              ctypes.byref(self.params), ctypes.c_void_p(self.workspace.data_ptr()),
                              int(nbytes.value), int(self.stream.cuda_stream))
        else:
            rc = L.sph_batch_create(ctypes.byref(self._h), len(self.cases), arr, ctypes.byref(self.params),
                                    ctypes.c_void_p(self.workspace.data_ptr()), int(nbytes.value),
                                    int(self.stream.cuda_stream))
        if rc != SPH_OK:
            raise SphError(rc, "sph_create failed (see stderr)")
        n_inst = ctypes.c_int32()
        npart = ctypes.c_int64()
        ncell = ctypes.c_int64()
        L.sph_sizes(self._h, ctypes.byref(n_inst), ctypes.byref(npart), ctypes.byref(ncell))
        self.n_inst, self.n, self.n_cells = n_inst.value, npart.value, ncell.value

    # -- helpers -------------------------------------------------------------
    def _check(self, rc):
        if rc != SPH_OK:
            msg = load().sph_last_error(self._h)
            raise SphError(rc, msg.decode() if msg else "")

    def close(self):
        if self._h:
            load().sph_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API -----------------------------------------------------------------
    def counts(self, inst=-1):
        out = np.zeros(4, np.int64)
        self._check(load().sph_counts(self._h, inst, out.ctypes.data_as(_I64)))
        return out

    def step(self, dt=0.0, nsteps=1):
        self._check(load().sph_step(self._h, float(dt), int(nsteps)))

    def sync(self):
        self._check(load().sph_sync(self._h))

    def probe_pressure(self, pts, inst=0):
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        out = np.zeros(pts.shape[0])
        self._check(load().sph_probe(self._h, inst, PROBE_PRESSURE, _d(pts), pts.shape[0], _d(out)))
        return out

    def probe_wave_height(self, xy, inst=0):
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        out = np.zeros(xy.shape[0])
        self._check(load().sph_probe(self._h, inst, PROBE_WAVE_HEIGHT, _d(xy), xy.shape[0], _d(out)))
        return out

    def probe_force(self, inst=0):
        out = np.zeros(3)
        self._check(load().sph_probe(self._h, inst, PROBE_FORCE, None, 0, _d(out)))
        return out

    def get_state(self):
        n = self.n
        r = np.zeros((n, 3)); u = np.zeros((n, 3)); rho = np.zeros(n); t = np.zeros(n, np.int32)
        up = np.zeros((n, 3)); rp = np.zeros(n); step = ctypes.c_int64(); time = np.zeros(self.n_inst)
        self._check(load().sph_get_state(self._h, _d(r), _d(u), _d(rho), t.ctypes.data_as(_I32), _d(up), _d(rp),
                                         ctypes.byref(step), _d(time)))
        return dict(r=r, u=u, rho=rho, type=t, uprev=up, rhoprev=rp, step=step.value, time=time)

    def time(self):
        """Physical time of every instance (only the clocks are copied)."""
        time = np.zeros(self.n_inst)
        step = ctypes.c_int64()
        self._check(load().sph_get_state(self._h, None, None, None, None, None, None, ctypes.byref(step),
                                         _d(time)))
        return time

    def set_state(self, r, u, rho, uprev=None, rhoprev=None, step=0, time=None):
        r = np.ascontiguousarray(r, np.float64); u = np.ascontiguousarray(u, np.float64)
        rho = np.ascontiguousarray(rho, np.float64)
        up = None if uprev is None else np.ascontiguousarray(uprev, np.float64)
        rp = None if rhoprev is None else np.ascontiguousarray(rhoprev, np.float64)
        tm = None if time is None else np.ascontiguousarray(np.broadcast_to(time, (self.n_inst,)), np.float64)
        assert r.shape == (self.n, 3) and u.shape == (self.n, 3) and rho.shape == (self.n,)
        self._check(load().sph_set_state(self._h, _d(r), _d(u), _d(rho), _opt(up, _d), _opt(rp, _d), int(step),
                                         _opt(tm, _d)))

    def checkpoint(self):
        """Host copy of the whole state (sph_get_state); restore() loads it
        into a handle of the same cases."""
        return self.get_state()

    def restore(self, ck):
        self.set_state(ck["r"], ck["u"], ck["rho"], ck["uprev"], ck["rhoprev"], ck["step"], ck["time"])

    def derivatives(self):
        n = self.n
        drho = np.zeros(n); acc = np.zeros((n, 3)); mu = np.zeros(n); nn = np.zeros(n, np.int32)
        self._check(load().sph_derivatives(self._h, _d(drho), _d(acc), _d(mu), nn.ctypes.data_as(_I32)))
        return drho, acc, mu, nn

    def cells(self):
        cell = np.zeros(self.n, np.int64); srt = np.zeros(self.n, np.int64)
        start = np.zeros(self.n_cells + 1, np.int64); nin = ctypes.c_int64()
        self._check(load().sph_cells(self._h, cell.ctypes.data_as(_I64), srt.ctypes.data_as(_I64),
                                     start.ctypes.data_as(_I64), ctypes.byref(nin)))
        return cell, srt[:nin.value], start

    def last_dt(self):
        out = np.zeros(self.n_inst)
        self._check(load().sph_last_dt(self._h, _d(out)))
        return out

    def diagnostics(self, inst=0):
        out = np.zeros(10)
        self._check(load().sph_diagnostics(self._h, inst, _d(out)))
        return out

    def set_profiling(self, on=True):
        self._check(load().sph_set_profiling(self._h, 1 if on else 0))

    def phase_times(self):
        L = load()
        k = L.sph_num_phases()
        ms = np.zeros(k); n = np.zeros(k, np.int64)
        self._check(L.sph_phase_times(self._h, _d(ms), n.ctypes.data_as(_I64), k))
        return {L.sph_phase_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(k)}

    def autotune(self, steps=3):
        """Tune cell size, pair launch shape and sort granularity; returns the
        pair shape (warps, CTAs per SM, particles per warp)."""
        best = np.zeros(3, np.int32)
        self._check(load().sph_autotune(self._h, int(steps), best.ctypes.data_as(_I32)))
        self._refresh_sizes()
        return tuple(int(v) for v in best)

    def tuned_config(self):
        out = np.zeros(5, np.int32)
        self._check(load().sph_tuned_config(self._h, out.ctypes.data_as(_I32)))
        return dict(pair_warps=int(out[0]), pair_ctas_per_sm=int(out[1]), pair_group=int(out[2]),
                    cell_div=int(out[3]), reorder_ctas_per_sm=int(out[4]))

    def _refresh_sizes(self):
        n_inst = ctypes.c_int32(); npart = ctypes.c_int64(); ncell = ctypes.c_int64()
        load().sph_sizes(self._h, ctypes.byref(n_inst), ctypes.byref(npart), ctypes.byref(ncell))
        self.n_cells = ncell.value

    def pair_stats(self):
        out = np.zeros(5, np.int64)
        self._check(load().sph_pair_stats(self._h, out.ctypes.data_as(_I64)))
        return dict(in_support=int(out[0]), evaluated=int(out[1]), candidates=int(out[2]),
                    fluid_fluid=int(out[3]), approaching=int(out[4]))

    def launches_per_step(self):
        return int(load().sph_launches_per_step(self._h))

    def list_stats(self):
        """Neighbour-list counters since the last call (list_skin > 0)."""
        out = np.zeros(4, np.int64)
        self._check(load().sph_list_stats(self._h, out.ctypes.data_as(_I64)))
        return dict(rebuilds=int(out[0]), reuses=int(out[1]), overflows=int(out[2]), longest=int(out[3]))

"""Plain FP64 CPU oracles of the WCSPH particle-interaction pass and of the MPS step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It compiles ``sph_oracle.c`` and ``mps_oracle.c`` with gcc into
``oracle/_build/liboracle.so`` and exposes its functions on numpy arrays.  It
shares no code with the CUDA library: the two meet only through plain arrays.

The method follows Section 2.2 of the paper (Eqs. 3-15) and the probes of
Sections 3.1-3.2 (Eq. 33); every reading of an open point is documented next to
the C code that takes it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_SRC_MPS = os.path.join(_HERE, "mps_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

FLUID, WALL, OBSTACLE, GATE = 0, 1, 2, 3
VERLET, SYMPLECTIC = 0, 1  # time integration: Eqs. 9-14, or the symplectic predictor-corrector
# delta term of Eq. 7: on every fluid particle (over its fluid neighbours), or
# off for a fluid particle that has a boundary neighbour
DELTA_ALL_FLUID, DELTA_FULL_SUPPORT = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction, OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_MPS))):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, _SRC_MPS, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, _SRC_MPS, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Case(ctypes.Structure):
    """Mirror of ``orc_case`` in sph_oracle.c."""

    _fields_ = [
        ("tank", ctypes.c_double * 3),
        ("column", ctypes.c_double * 3),
        ("has_obstacle", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("obstacle", ctypes.c_double * 6),
        ("dp", ctypes.c_double),
        ("h", ctypes.c_double),
        ("c0", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("g", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("ns", ctypes.c_int32),
        ("layers", ctypes.c_int32),
        ("init_mode", ctypes.c_int32),
        ("csound_mode", ctypes.c_int32),
        ("cell_div", ctypes.c_int32),
        ("integrator", ctypes.c_int32),
        ("has_gate", ctypes.c_int32),
        ("delta_mode", ctypes.c_int32),
        ("gate", ctypes.c_double * 6),
        ("gate_v", ctypes.c_double * 3),
    ]


def make_case(tank, column, obstacle=None, *, dp, h, c0, rho0=1000.0, alpha=0.01, gamma=7.0,
              g=9.81, delta=0.1, cfl=0.2, ns=40, layers=2, init_mode=0, csound_mode=0,
              cell_div=2, integrator=VERLET, gate=None, gate_velocity=(0.0, 0.0, 0.0),
              delta_mode=DELTA_ALL_FLUID) -> Case:
    c = Case()
    c.tank[:] = [float(v) for v in tank]
    c.column[:] = [float(v) for v in column]
    c.has_obstacle = 0 if obstacle is None else 1
    if obstacle is not None:
        c.obstacle[:] = [float(v) for v in obstacle]
    c.dp, c.h, c.c0, c.rho0, c.alpha = dp, h, c0, rho0, alpha
    c.gamma, c.g, c.delta, c.cfl = gamma, g, delta, cfl
    c.ns, c.layers, c.init_mode, c.csound_mode, c.cell_div = ns, layers, init_mode, csound_mode, cell_div
    c.integrator = integrator
    c.delta_mode = delta_mode
    if gate is not None:
        c.has_gate = 1
        c.gate[:] = [float(v) for v in gate]
        c.gate_v[:] = [float(v) for v in gate_velocity]
    return c


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_CP = ctypes.POINTER(Case)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_kernel_w": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
                "orc_kernel_dwdr": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
                "orc_kernel_f": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
                "orc_tait": (ctypes.c_double, [_CP, ctypes.c_double]),
                "orc_sound": (ctypes.c_double, [_CP, ctypes.c_double]),
                "orc_nu0": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int]),
                "orc_scene_counts": (ctypes.c_int, [_CP, _I64]),
                "orc_scene_build": (ctypes.c_int, [_CP, _D, _D, _D, _I32]),
                "orc_grid_info": (None, [_CP, _D, _D, _I64]),
                "orc_num_cells": (ctypes.c_int64, [_CP]),
                "orc_cells": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _I64, _I64, _I64]),
                "orc_neighbour_counts": (ctypes.c_int, [_CP, ctypes.c_int64, _D, ctypes.c_int, _I32]),
                "orc_derivatives": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _I32, _D, _D, _D,
                                                   _I32]),
                "orc_derivatives_subset": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _I32,
                                                          ctypes.c_int64, _I64, _D, _D, _D, _I32]),
                "orc_dt": (ctypes.c_double, [_CP, ctypes.c_int64, _I32, _I32, _D, _D]),
                "orc_step": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _D, _D, _I32,
                                            ctypes.c_int64, ctypes.c_double, _D]),
                "orc_run": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _D, _D, _I32,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _D]),
                "orc_probe_pressure": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _I32,
                                                      ctypes.c_int64, _D, _D]),
                "orc_probe_wave_height": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _I32,
                                                         ctypes.c_int64, _D, _D]),
                "orc_probe_force": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _I32, _D]),
                "orc_diagnostics": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _I32, _D]),
                "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i32(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


def _i64(a):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_I64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def kernel_w(r, h):
    return lib().orc_kernel_w(float(r), float(h))


def kernel_dwdr(r, h):
    return lib().orc_kernel_dwdr(float(r), float(h))


def kernel_f(r, h):
    return lib().orc_kernel_f(float(r), float(h))


def tait(case, rho):
    return lib().orc_tait(ctypes.byref(case), float(rho))


def sound(case, rho):
    return lib().orc_sound(ctypes.byref(case), float(rho))


def nu0(alpha, h, c0, dim=3):
    return lib().orc_nu0(float(alpha), float(h), float(c0), int(dim))


class State:
    """Particle state in id order: r (n,3), u (n,3), rho (n), previous level, type."""

    def __init__(self, r, u, rho, type_, uprev=None, rhoprev=None, step=0):
        self.r = np.ascontiguousarray(r, dtype=np.float64)
        self.u = np.ascontiguousarray(u, dtype=np.float64)
        self.rho = np.ascontiguousarray(rho, dtype=np.float64)
        self.type = np.ascontiguousarray(type_, dtype=np.int32)
        self.uprev = np.array(self.u if uprev is None else uprev, dtype=np.float64, order="C")
        self.rhoprev = np.array(self.rho if rhoprev is None else rhoprev, dtype=np.float64, order="C")
        self.step = int(step)

    @property
    def n(self):
        return self.rho.shape[0]

    def copy(self):
        return State(self.r.copy(), self.u.copy(), self.rho.copy(), self.type.copy(), self.uprev.copy(),
                     self.rhoprev.copy(), self.step)


def scene_counts(case):
    c = np.zeros(3, np.int64)
    _check(lib().orc_scene_counts(ctypes.byref(case), _i64(c)), "scene_counts")
    return c


def scene(case) -> State:
    n = int(scene_counts(case).sum())
    r = np.zeros((n, 3)); u = np.zeros((n, 3)); rho = np.zeros(n); t = np.zeros(n, np.int32)
    _check(lib().orc_scene_build(ctypes.byref(case), _d(r), _d(u), _d(rho), _i32(t)), "scene_build")
    return State(r, u, rho, t)


def grid_info(case):
    lo = np.zeros(3); size = ctypes.c_double(); dims = np.zeros(3, np.int64)
    lib().orc_grid_info(ctypes.byref(case), _d(lo), ctypes.byref(size), _i64(dims))
    return lo, size.value, dims


def cells(case, r):
    """(cell[n], order[n], start[ncells + 2]) of the counting sort by cell."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = r.shape[0]
    ncells = lib().orc_num_cells(ctypes.byref(case))
    cell = np.zeros(n, np.int64); order = np.zeros(n, np.int64); start = np.zeros(ncells + 2, np.int64)
    _check(lib().orc_cells(ctypes.byref(case), n, _d(r), _i64(cell), _i64(order), _i64(start)), "cells")
    return cell, order, start


def neighbour_counts(case, r, brute=False):
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(r.shape[0], np.int32)
    _check(lib().orc_neighbour_counts(ctypes.byref(case), r.shape[0], _d(r), 1 if brute else 0, _i32(out)),
           "neighbour_counts")
    return out


def derivatives(case, st: State):
    n = st.n
    drho = np.zeros(n); acc = np.zeros((n, 3)); mumax = np.zeros(n); nn = np.zeros(n, np.int32)
    _check(lib().orc_derivatives(ctypes.byref(case), n, _d(st.r), _d(st.u), _d(st.rho), _i32(st.type),
                                 _d(drho), _d(acc), _d(mumax), _i32(nn)), "derivatives")
    return drho, acc, mumax, nn


def derivatives_subset(case, st: State, sel):
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    k = sel.shape[0]
    drho = np.zeros(k); acc = np.zeros((k, 3)); mumax = np.zeros(k); nn = np.zeros(k, np.int32)
    _check(lib().orc_derivatives_subset(ctypes.byref(case), st.n, _d(st.r), _d(st.u), _d(st.rho),
                                        _i32(st.type), k, _i64(sel), _d(drho), _d(acc), _d(mumax), _i32(nn)),
           "derivatives_subset")
    return drho, acc, mumax, nn


def dt(case, type_, nneigh, acc, mumax):
    return lib().orc_dt(ctypes.byref(case), type_.shape[0], _i32(np.ascontiguousarray(type_, np.int32)),
                        _i32(np.ascontiguousarray(nneigh, np.int32)),
                        _d(np.ascontiguousarray(acc, np.float64)), _d(np.ascontiguousarray(mumax, np.float64)))


def step(case, st: State, dt_fixed=0.0):
    """Advance ``st`` in place by one step; returns the dt used."""
    used = ctypes.c_double()
    _check(lib().orc_step(ctypes.byref(case), st.n, _d(st.r), _d(st.u), _d(st.rho), _d(st.uprev),
                          _d(st.rhoprev), _i32(st.type), st.step, float(dt_fixed), ctypes.byref(used)), "step")
    st.step += 1
    return used.value


def run(case, st: State, nsteps, dt_fixed=0.0):
    """Advance ``st`` in place by ``nsteps`` steps; returns the dts."""
    dts = np.zeros(max(int(nsteps), 1))
    _check(lib().orc_run(ctypes.byref(case), st.n, _d(st.r), _d(st.u), _d(st.rho), _d(st.uprev),
                         _d(st.rhoprev), _i32(st.type), st.step, int(nsteps), float(dt_fixed), _d(dts)), "run")
    st.step += int(nsteps)
    return dts[:int(nsteps)]


def probe_pressure(case, st: State, pts):
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(pts.shape[0])
    _check(lib().orc_probe_pressure(ctypes.byref(case), st.n, _d(st.r), _d(st.rho), _i32(st.type),
                                    pts.shape[0], _d(pts), _d(out)), "probe_pressure")
    return out


def probe_wave_height(case, st: State, pts_xy):
    pts = np.ascontiguousarray(pts_xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(pts.shape[0])
    _check(lib().orc_probe_wave_height(ctypes.byref(case), st.n, _d(st.r), _i32(st.type), pts.shape[0],
                                       _d(pts), _d(out)), "probe_wave_height")
    return out


def probe_force(case, st: State):
    out = np.zeros(3)
    _check(lib().orc_probe_force(ctypes.byref(case), st.n, _d(st.r), _d(st.u), _d(st.rho), _i32(st.type),
                                 _d(out)), "probe_force")
    return out


def diagnostics(case, st: State):
    out = np.zeros(10)
    _check(lib().orc_diagnostics(ctypes.byref(case), st.n, _d(st.r), _d(st.u), _d(st.rho), _i32(st.type),
                                 _d(out)), "diagnostics")
    return out

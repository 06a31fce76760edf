"""Plain FP64 CPU oracle of one MPS step (test infrastructure; ``mps_oracle.c``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It follows Section 2.3 of the paper
(Eqs. 16-30) with the parameters of Section 3; every reading of an open point
is documented next to the C code that takes it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib as _lib_sph

FLUID, WALL, DUMMY = 0, 1, 2


class MpsCase(ctypes.Structure):
    """Mirror of ``mps_case`` in mps_oracle.c."""

    _fields_ = [
        ("tank", ctypes.c_double * 3),
        ("column", ctypes.c_double * 3),
        ("l0", ctypes.c_double),
        ("re", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("g", ctypes.c_double),
        ("kappa_c", ctypes.c_double),
        ("kappa_r", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("varrho1", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("cg_tol", ctypes.c_double),
        ("layers", ctypes.c_int32),
        ("cg_max", ctypes.c_int32),
    ]


def make_case(tank, column, *, l0, dt, re_factor=2.1, nu=1e-6, rho=1000.0, g=9.81, kappa_c=1e-8, kappa_r=0.01,
              beta1=0.98, varrho1=0.2, cg_tol=1e-6, layers=3, cg_max=100000) -> MpsCase:
    c = MpsCase()
    c.tank[:] = [float(v) for v in tank]
    c.column[:] = [float(v) for v in column]
    c.l0, c.re, c.nu, c.rho, c.g = l0, re_factor * l0, nu, rho, g
    c.kappa_c, c.kappa_r, c.beta1, c.varrho1, c.dt, c.cg_tol = kappa_c, kappa_r, beta1, varrho1, dt, cg_tol
    c.layers, c.cg_max = layers, cg_max
    return c


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_CP = ctypes.POINTER(MpsCase)
_bound = False


def lib():
    global _bound
    L = _lib_sph()
    if not _bound:
        sig = {
            "mps_weight": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "mps_lattice_constants": (None, [_CP, _D, _D]),
            "mps_scene_counts": (ctypes.c_int, [_CP, _I64]),
            "mps_scene_build": (ctypes.c_int, [_CP, _D, _I32]),
            "mps_pnd": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D]),
            "mps_operators": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _D, _D]),
            "mps_step": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _D, _I32, _D, _D, _I32, _D]),
            "mps_pressure": (ctypes.c_int, [_CP, ctypes.c_int64, _D, _I32, _D, _D, _I32, _D, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i32(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"MPS oracle {what} failed ({rc})")


def weight(r, re):
    return lib().mps_weight(float(r), float(re))


def lattice_constants(case):
    n0 = ctypes.c_double()
    lam = ctypes.c_double()
    lib().mps_lattice_constants(ctypes.byref(case), ctypes.byref(n0), ctypes.byref(lam))
    return n0.value, lam.value


def scene(case):
    c = np.zeros(3, np.int64)
    _check(lib().mps_scene_counts(ctypes.byref(case), c.ctypes.data_as(_I64)), "scene_counts")
    n = int(c.sum())
    r = np.zeros((n, 3))
    t = np.zeros(n, np.int32)
    _check(lib().mps_scene_build(ctypes.byref(case), _d(r), _i32(t)), "scene_build")
    return r, t


def pnd(case, r):
    r = np.ascontiguousarray(r, np.float64)
    out = np.zeros(r.shape[0])
    _check(lib().mps_pnd(ctypes.byref(case), r.shape[0], _d(r), _d(out)), "pnd")
    return out


def operators(case, r, phi):
    r = np.ascontiguousarray(r, np.float64)
    phi = np.ascontiguousarray(phi, np.float64)
    grad = np.zeros((r.shape[0], 3))
    lap = np.zeros(r.shape[0])
    _check(lib().mps_operators(ctypes.byref(case), r.shape[0], _d(r), _d(phi), _d(grad), _d(lap)), "operators")
    return grad, lap


def pressure(case, r, type_):
    r = np.ascontiguousarray(r, np.float64)
    t = np.ascontiguousarray(type_, np.int32)
    n = r.shape[0]
    P = np.zeros(n); nd = np.zeros(n); surf = np.zeros(n, np.int32); sigma = np.zeros(n); cg = np.zeros(2)
    _check(lib().mps_pressure(ctypes.byref(case), n, _d(r), _i32(t), _d(P), _d(nd), _i32(surf), _d(sigma),
                              _d(cg)), "pressure")
    return dict(P=P, nd=nd, surf=surf, sigma=sigma, iterations=int(cg[0]), residual=float(cg[1]))


def step(case, r, u, type_):
    """One MPS step; r and u (n, 3) are advanced in place."""
    t = np.ascontiguousarray(type_, np.int32)
    n = r.shape[0]
    P = np.zeros(n); nd = np.zeros(n); surf = np.zeros(n, np.int32); cg = np.zeros(2)
    _check(lib().mps_step(ctypes.byref(case), n, _d(r), _d(u), _i32(t), _d(P), _d(nd), _i32(surf), _d(cg)),
           "step")
    return dict(P=P, nd=nd, surf=surf, iterations=int(cg[0]), residual=float(cg[1]))

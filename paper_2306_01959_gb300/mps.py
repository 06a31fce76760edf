"""Python binding of the MPS entry points of ``include/mps.h`` (argument
marshalling only; every step runs in ``libsph.so``).  PyTorch provides the
device workspace and the stream."""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import sph

FLUID, WALL, DUMMY = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("layers", ctypes.c_int32),
        ("re_factor", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("g", ctypes.c_double),
        ("kappa_c", ctypes.c_double),
        ("kappa_r", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("varrho1", ctypes.c_double),
        ("cg_tol", ctypes.c_double),
        ("cg_max", ctypes.c_int32),
        ("row_width", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p

SIGNATURES = {
    "mps_params_default": (None, [ctypes.POINTER(Params)]),
    "mps_workspace_size": (ctypes.c_int, [_D, _D, ctypes.c_double, ctypes.POINTER(Params),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "mps_create": (ctypes.c_int, [ctypes.POINTER(_VP), _D, _D, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(Params), _VP, ctypes.c_size_t, ctypes.c_size_t]),
    "mps_destroy": (None, [_VP]),
    "mps_step": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "mps_pressure": (ctypes.c_int, [_VP, _D, _D, _I32, _I64, _D]),
    "mps_get_state": (ctypes.c_int, [_VP, _D, _D, _D, _I32, _I64]),
    "mps_set_state": (ctypes.c_int, [_VP, _D, _D]),
    "mps_last_solve": (ctypes.c_int, [_VP, _I64, _D]),
    "mps_counts": (ctypes.c_int, [_VP, _I64]),
    "mps_system_size": (ctypes.c_int, [_VP, _I64]),
    "mps_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "mps_phase_times": (ctypes.c_int, [_VP, _D]),
    "mps_last_error": (ctypes.c_char_p, [_VP]),
}

_bound = False


def load():
    global _bound
    L = sph.load()
    if not _bound:
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def default_params(**kw) -> Params:
    p = Params()
    load().mps_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _arr3(v):
    return (ctypes.c_double * 3)(*[float(x) for x in v])


class Tank:
    """One MPS dam-break tank (a handle of include/mps.h)."""

    def __init__(self, tank, column, l0, dt, params: Optional[Params] = None, device="cuda", **kw):
        import torch

        L = load()
        self.params = params if params is not None else default_params(**kw)
        t3, c3 = _arr3(tank), _arr3(column)
        nbytes = ctypes.c_size_t()
        rc = L.mps_workspace_size(t3, c3, float(l0), ctypes.byref(self.params), ctypes.byref(nbytes))
        if rc != sph.SPH_OK:
            raise sph.SphError(rc, "invalid MPS tank or parameters")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.workspace.device)
        self._h = _VP()
        rc = L.mps_create(ctypes.byref(self._h), t3, c3, float(l0), float(dt), ctypes.byref(self.params),
                          ctypes.c_void_p(self.workspace.data_ptr()), int(nbytes.value), int(self.stream.cuda_stream))
        if rc != sph.SPH_OK:
            raise sph.SphError(rc, "mps_create failed")
        out = np.zeros(4, np.int64)
        L.mps_counts(self._h, out.ctypes.data_as(_I64))
        self.counts = out
        self.n = int(out[3])

    def _check(self, rc):
        if rc != sph.SPH_OK:
            msg = load().mps_last_error(self._h)
            raise sph.SphError(rc, msg.decode() if msg else "")

    def close(self):
        if self._h:
            load().mps_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        self._check(load().mps_step(self._h, int(nsteps)))

    def pressure(self):
        n = self.n
        P = np.zeros(n); nd = np.zeros(n); surf = np.zeros(n, np.int32)
        it = ctypes.c_int64(); res = ctypes.c_double()
        self._check(load().mps_pressure(self._h, P.ctypes.data_as(_D), nd.ctypes.data_as(_D),
                                        surf.ctypes.data_as(_I32), ctypes.byref(it), ctypes.byref(res)))
        return dict(P=P, nd=nd, surf=surf, iterations=it.value, residual=res.value)

    def get_state(self):
        n = self.n
        r = np.zeros((n, 3)); u = np.zeros((n, 3)); P = np.zeros(n); t = np.zeros(n, np.int32)
        step = ctypes.c_int64()
        self._check(load().mps_get_state(self._h, r.ctypes.data_as(_D), u.ctypes.data_as(_D), P.ctypes.data_as(_D),
                                         t.ctypes.data_as(_I32), ctypes.byref(step)))
        return dict(r=r, u=u, P=P, type=t, step=step.value)

    def set_state(self, r, u):
        r = np.ascontiguousarray(r, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        assert r.shape == (self.n, 3) and u.shape == (self.n, 3)
        self._check(load().mps_set_state(self._h, r.ctypes.data_as(_D), u.ctypes.data_as(_D)))

    def set_profiling(self, on=True):
        self._check(load().mps_set_profiling(self._h, 1 if on else 0))

    def phase_times(self):
        ms = np.zeros(4)
        self._check(load().mps_phase_times(self._h, ms.ctypes.data_as(_D)))
        return dict(zip(("neighbours_prediction", "density_assembly", "cg", "gradient_correction"),
                        ms.tolist()))

    def system_size(self):
        """Rows and stored off-diagonal entries of the last Eq. 23 system."""
        out = np.zeros(2, np.int64)
        self._check(load().mps_system_size(self._h, out.ctypes.data_as(_I64)))
        return int(out[0]), int(out[1])

    def last_solve(self):
        it = ctypes.c_int64(); res = ctypes.c_double()
        self._check(load().mps_last_solve(self._h, ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

"""Pins of the MPS oracle (Section 2.3) against what the paper and the
mathematics fix: the weight function and its support, the lattice constants
n0 and lambda0 by direct enumeration, the gradient and Laplacian operators on
linear and quadratic fields, the free-surface criteria by brute force, the CG
solution against an independently assembled system, and a still column whose
time-averaged pressure is hydrostatic.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mps as M

L0 = 0.02


def case(**kw):
    kw.setdefault("dt", 3e-4)
    return M.make_case((0.24, 0.24, 0.4), (0.24, 0.24, 0.3), l0=L0, **kw)


def block(n=9, origin=(0.05, 0.05, 0.05)):
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.asarray(origin) + L0 * np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)


def test_weight_function_eq16():
    re = 2.1 * L0
    assert M.weight(re / 2, re) == pytest.approx(1.0, abs=1e-15)
    assert M.weight(re, re) == 0.0  # continuous at r_e
    assert M.weight(1.01 * re, re) == 0.0  # zero beyond r_e (the printed "> 0" read as "> r_e")
    assert M.weight(L0, re) == pytest.approx(1.1, abs=1e-14)
    assert M.weight(0.0, re) == 0.0  # coincident particles are not neighbours


def test_lattice_constants_by_enumeration():
    c = case()
    n0, lam = M.lattice_constants(c)
    re = 2.1 * L0
    pts = [(a, b, d) for a in range(-3, 4) for b in range(-3, 4) for d in range(-3, 4) if (a, b, d) != (0, 0, 0)]
    r = np.array([L0 * math.sqrt(a * a + b * b + d * d) for a, b, d in pts])
    w = np.where(r <= re, re / r - 1.0, 0.0)
    assert np.count_nonzero(w) == 32  # |d|^2 in {1, 2, 3, 4} within 2.1 l0
    assert n0 == pytest.approx(w.sum(), rel=1e-14)
    assert lam == pytest.approx((r * r * w).sum() / w.sum(), rel=1e-14)
    # the 32 neighbours: 6 at l0, 12 at sqrt2 l0, 8 at sqrt3 l0, 6 at 2 l0
    assert n0 == pytest.approx(6 * 1.1 + 12 * (2.1 / math.sqrt(2) - 1) + 8 * (2.1 / math.sqrt(3) - 1) + 6 * 0.05,
                               rel=1e-14)


def test_operators_on_linear_and_quadratic_fields():
    # On a full lattice neighbourhood the gradient of Eq. 18 is exact for a
    # linear field, and the Laplacian of Eq. 19 (with lambda0 of Eq. 20) gives
    # 2 for x^2 and 6 for |r|^2.
    c = case()
    r = block()
    centre = np.all(np.abs(r - r.mean(axis=0)) < 1.5 * L0, axis=1)
    a = np.array([0.3, -1.2, 2.5])
    grad, _ = M.operators(c, r, r @ a)
    assert np.allclose(grad[centre], a, rtol=0, atol=1e-12)
    _, lap = M.operators(c, r, r[:, 0] ** 2)
    assert np.allclose(lap[centre], 2.0, rtol=1e-12)
    _, lap = M.operators(c, r, (r ** 2).sum(axis=1))
    assert np.allclose(lap[centre], 6.0, rtol=1e-12)
    nd = M.pnd(c, r)
    n0, _ = M.lattice_constants(c)
    assert np.allclose(nd[centre], n0, rtol=1e-14)


def test_free_surface_criteria_by_brute_force():
    c = case()
    r, t = M.scene(c)
    rng = np.random.Generator(np.random.PCG64(3))
    f = t == M.FLUID
    r = r.copy()
    r[f] += rng.normal(0.0, 0.05 * L0, (int(f.sum()), 3))
    out = M.pressure(c, r, t)
    n0, _ = M.lattice_constants(c)
    re = 2.1 * L0
    d = r[None, :, :] - r[:, None, :]
    dist = np.sqrt((d ** 2).sum(axis=2))
    w = np.where((dist > 0) & (dist <= re), re / np.where(dist > 0, dist, 1.0) - 1.0, 0.0)
    nd = w.sum(axis=1)
    assert np.allclose(out["nd"], nd, rtol=1e-12)
    sig = np.sqrt(((d * w[:, :, None]).sum(axis=1) ** 2).sum(axis=1)) / np.where(nd > 0, nd, 1.0)
    surf = (t != M.DUMMY) & (nd < 0.98 * n0) & (sig > 0.2 * L0)
    assert np.array_equal(out["surf"].astype(bool), surf)
    # the top fluid layer is free surface, the fluid under it is not
    top = f & (r[:, 2] > 0.3 - L0)
    deep = f & (r[:, 2] < 0.3 - 3 * L0) & np.all(np.abs(r[:, :2] - 0.12) < 0.06, axis=1)
    assert surf[top].mean() > 0.95 and not surf[deep].any()


def test_cg_solution_of_an_independently_assembled_ppe():
    # Eq. 23 assembled here from its definition (dense, brute force): unknowns
    # are the fluid and wall particles off the free surface; a free-surface
    # neighbour has P = 0; dummy particles take no part.  The oracle's CG
    # solution must leave a relative residual <= 1e-6 in this system.
    c = case()
    r, t = M.scene(c)
    rng = np.random.Generator(np.random.PCG64(5))
    f = t == M.FLUID
    r = r.copy()
    r[f] += rng.normal(0.0, 0.05 * L0, (int(f.sum()), 3))
    r[f, 2] -= 0.02 * L0 * (0.3 - r[f, 2]) / 0.3  # compress the column towards the floor
    out = M.pressure(c, r, t)
    n0, lam = M.lattice_constants(c)
    re = 2.1 * L0
    unknown = (t != M.DUMMY) & (out["surf"] == 0)
    idx = np.flatnonzero(unknown)
    ru = r[idx]
    d = np.sqrt(((r[idx][:, None, :] - r[None, :, :]) ** 2).sum(axis=2))
    w = np.where((d > 0) & (d <= re), re / np.where(d > 0, d, 1.0) - 1.0, 0.0)
    w[:, t == M.DUMMY] = 0.0
    cc = 6.0 / (lam * n0)
    kc = 1000.0 * 1e-8 / c.dt ** 2
    A = -cc * w[:, idx]
    A[np.arange(len(idx)), np.arange(len(idx))] = cc * w.sum(axis=1) + kc
    b = 0.01 * 1000.0 / c.dt ** 2 * (out["nd"][idx] - n0) / n0
    x = out["P"][idx]
    assert np.allclose(A, A.T, rtol=0, atol=1e-9 * cc)
    assert np.linalg.norm(A @ x - b) <= 1.0001e-6 * np.linalg.norm(b)
    assert out["residual"] <= 1e-6 and out["iterations"] > 5
    exact = np.linalg.solve(A, b)
    assert np.linalg.norm(x - exact) <= 1e-3 * np.linalg.norm(exact)
    assert np.all(out["P"][~unknown] == 0.0)


def test_still_column_time_averaged_pressure_is_hydrostatic():
    # A still column (0.3 m deep, l0 = 0.02 m, dt = 3e-4 s) started at rest
    # oscillates about its equilibrium under the relaxed source of Eq. 23; the
    # pressure averaged over steps 500-1500 has the hydrostatic gradient
    # rho g within 2 %, vanishes at the free-surface layer (within l0/2), and
    # is rho g (z0 - z) within 3 % at interior points.
    c = case()
    r, t = M.scene(c)
    u = np.zeros_like(r)
    threads = oracle.set_threads(8)
    f = t == M.FLUID
    inner = np.flatnonzero(f & (np.abs(r[:, 0] - 0.13) < 0.011) & (np.abs(r[:, 1] - 0.13) < 0.011))
    acc = []
    for k in range(1500):
        out = M.step(c, r, u, t)
        if k >= 500:
            acc.append(out["P"][inner])
    oracle.set_threads(threads)
    z = r[inner, 2]
    p = np.mean(acc, axis=0) / (1000.0 * 9.81)
    zf = r[f, 2]
    ztop = zf[zf > zf.max() - 0.5 * L0].mean()
    sel = (z > 0.04) & (z < ztop - 0.05)
    a, b0 = np.polyfit(z[sel], p[sel], 1)
    z0 = -b0 / a
    assert abs(-a - 1.0) <= 0.02, a
    assert abs(z0 - ztop) <= 0.5 * L0, (z0, ztop)
    assert np.all(np.abs(p[sel] / (z0 - z[sel]) - 1.0) <= 0.03)

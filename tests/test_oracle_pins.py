"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a quadrature, a
closed form, an invariant, a brute-force count, or a value printed in the paper.
A dropped term, a wrong sign or factor, or a transposed index in the oracle makes
at least one of them fail.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2306_01959_gb300 import workloads as wl

HF = 1.2 * math.sqrt(3.0)


def big_case(dp=0.02, h=None, **kw):
    """A case whose grid comfortably holds free-standing lattice blocks."""
    h = HF * dp if h is None else h
    kw.setdefault("c0", 10.0 * math.sqrt(9.81 * 0.3))
    return oracle.make_case((2.0, 2.0, 2.0), (0.0, 0.0, 0.0), dp=dp, h=h, **kw)


def lattice(n, dp, origin=(0.5, 0.5, 0.5)):
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    return np.asarray(origin, np.float64) + (pts + 0.5) * dp


def fluid_state(r, rho=1000.0, u=None):
    n = r.shape[0]
    return oracle.State(r, np.zeros((n, 3)) if u is None else u, np.full(n, rho) if np.isscalar(rho) else rho,
                        np.zeros(n, np.int32))


# ---------------------------------------------------------------- Eq. 6 kernel
@pytest.mark.parametrize("h", [0.01, 0.0207846, 0.5])
def test_wendland_normalises_to_one(h):
    # Eq. 6 with the 3D constant read as 21/(16 pi h^3): int W dV = 1.
    val, _ = integrate.quad(lambda r: 4.0 * math.pi * r * r * oracle.kernel_w(r, h), 0.0, 2.0 * h,
                            epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("h", [0.01, 0.3])
def test_gradient_second_moment_is_minus_identity(h):
    # int x_a d_b W dV = -delta_ab; with grad W = F(r) x this is (4 pi / 3) int r^4 F dr = -1.
    val, _ = integrate.quad(lambda r: 4.0 * math.pi / 3.0 * r ** 4 * oracle.kernel_f(r, h), 0.0, 2.0 * h,
                            epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val + 1.0) < 1e-10


def test_gradient_matches_finite_difference():
    h = 0.02
    for q in [0.05, 0.3, 0.9, 1.3, 1.77, 1.99]:
        r = q * h
        eps = 1e-7 * h
        fd = (oracle.kernel_w(r + eps, h) - oracle.kernel_w(r - eps, h)) / (2 * eps)
        assert abs(oracle.kernel_dwdr(r, h) - fd) <= 1e-6 * abs(fd) + 1e-9
        assert abs(oracle.kernel_f(r, h) * r - fd) <= 1e-6 * abs(fd) + 1e-9
    assert oracle.kernel_w(2.0 * h, h) == 0.0 and oracle.kernel_f(2.0 * h, h) == 0.0
    assert oracle.kernel_w(3.0 * h, h) == 0.0


# ---------------------------------------------------------------- Eq. 8 EOS
def test_tait_eos_and_sound_speed():
    case = big_case()
    assert oracle.tait(case, 1000.0) == 0.0
    for rho in [985.0, 1000.0, 1003.0, 1030.0]:
        d = 1e-4
        dpdrho = (oracle.tait(case, rho + d) - oracle.tait(case, rho - d)) / (2 * d)
        c = oracle.sound(case, rho)
        assert abs(c * c - dpdrho) < 1e-6 * dpdrho
    # gamma = 1 makes Eq. 8 linear: P = c0^2 (rho - rho0)
    lin = big_case(gamma=1.0)
    assert abs(oracle.tait(lin, 1010.0) - lin.c0 ** 2 * 10.0) < 1e-8


# ---------------------------------------------------------------- Eq. 32 against Tables 1 and 3
def test_nu0_alpha_relation_matches_printed_tables():
    path = os.path.join(os.path.dirname(__file__), "golden", "nu0_alpha_tables.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 7
    for alpha, l0, hw, printed, digits in rows:
        alpha, l0, hw, printed, digits = float(alpha), float(l0), float(hw), float(printed), int(digits)
        h = 1.5 * l0
        c0 = 20.0 * math.sqrt(9.81 * hw)
        val = oracle.nu0(alpha, h, c0, 3)
        rounded = float(f"{val:.{digits - 1}e}")
        assert rounded == printed, (alpha, l0, val, printed)


# ---------------------------------------------------------------- neighbour structure
def _lattice_count(k):
    m = int(math.ceil(k))
    v = np.arange(-m, m + 1)
    x, y, z = np.meshgrid(v, v, v, indexing="ij")
    d2 = x * x + y * y + z * z
    return int(np.count_nonzero((d2 < k * k) & (d2 > 0)))


@pytest.mark.parametrize("hfac,cell_div", [(HF, 1), (HF, 2), (1.55, 1), (1.55, 3)])
def test_interior_lattice_neighbour_count(hfac, cell_div):
    # 2h/dp is kept off lattice distances (2h = 3 dp would put 30 lattice points
    # exactly on the support edge, where rounding decides).
    dp = 0.02
    case = big_case(dp, hfac * dp, cell_div=cell_div)
    r = lattice(11, dp)
    nn = oracle.neighbour_counts(case, r)
    centre = 5 + 11 * (5 + 11 * 5)
    assert nn[centre] == _lattice_count(2.0 * hfac)
    assert _lattice_count(2.0 * HF) == 304 and _lattice_count(3.0) == 92


@pytest.mark.parametrize("cell_div", [1, 2, 3])
def test_cell_list_equals_brute_force(cell_div):
    dp = 0.02
    case = big_case(dp, cell_div=cell_div)
    rng = np.random.Generator(np.random.PCG64(11 + cell_div))
    r = rng.uniform(-0.1, 0.4, size=(700, 3))
    r[:5] = [[-0.5, 0.1, 0.1], [0.1, 2.5, 0.1], [0.1, 0.1, 9.0], [0.0, 0.0, 0.0], [0.2, 0.2, 0.2]]
    r[5] = r[4]  # a coincident pair
    a = oracle.neighbour_counts(case, r)
    b = oracle.neighbour_counts(case, r, brute=True)
    assert np.array_equal(a, b)
    assert (a[:3] == -1).all() and a[4] >= 1


def test_counting_sort_order_and_cells():
    dp = 0.02
    case = big_case(dp, cell_div=2)
    rng = np.random.Generator(np.random.PCG64(3))
    r = rng.uniform(-0.2, 2.3, size=(3000, 3))
    cell, order, start = oracle.cells(case, r)
    lo, size, dims = oracle.grid_info(case)
    ncells = int(np.prod(dims))
    # cell ids recomputed independently from the grid description
    c = np.floor((r - lo) / size)
    inside = np.all((c >= 0) & (c < dims), axis=1)
    lin = (c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]
    expect = np.where(inside, lin, ncells).astype(np.int64)
    assert np.array_equal(cell, expect)
    # ascending (cell, id) order, the starts bracket each cell
    key = cell[order] * len(r) + order
    assert np.all(np.diff(key) > 0)
    for cc in np.unique(cell):
        assert np.array_equal(np.sort(order[start[cc]:start[cc + 1]]), np.flatnonzero(cell == cc))


# ---------------------------------------------------------------- Eq. 7
def test_uniform_compression_raises_density():
    # u = -eps (r - c): div u = -3 eps, so D rho/Dt = -rho div u = 3 eps rho0 inside.
    dp = 0.02
    case = big_case(dp, delta=0.0)
    r = lattice(13, dp)
    c = r.mean(axis=0)
    eps = 0.5
    st = fluid_state(r, u=-eps * (r - c))
    drho, acc, mumax, nn = oracle.derivatives(case, st)
    centre = np.argmin(np.linalg.norm(r - c, axis=1))
    assert drho[centre] > 0
    assert abs(drho[centre] / (3 * eps * 1000.0) - 1.0) < 0.02


def test_delta_term_is_delta_h_c0_laplacian():
    # With u = 0 only the delta term of Eq. 7 remains; for rho = rho0 + k x^2 it
    # approximates delta h c0 lap(rho) = 2 k delta h c0.  A constant rho gives 0.
    dp = 0.02
    case = big_case(dp, delta=0.1)
    r = lattice(13, dp)
    c = r.mean(axis=0)
    centre = np.argmin(np.linalg.norm(r - c, axis=1))
    kx = 50.0
    rho = 1000.0 + kx * (r[:, 0] - c[0]) ** 2
    drho, *_ = oracle.derivatives(case, fluid_state(r, rho=rho))
    expect = 2.0 * kx * 0.1 * case.h * case.c0
    assert abs(drho[centre] / expect - 1.0) < 0.03
    drho0, *_ = oracle.derivatives(case, fluid_state(r, rho=1003.0))
    assert np.max(np.abs(drho0)) == 0.0
    # delta = 0 removes the term
    drho_off, *_ = oracle.derivatives(big_case(dp, delta=0.0), fluid_state(r, rho=rho))
    assert np.max(np.abs(drho_off)) == 0.0


# ---------------------------------------------------------------- Eq. 3 invariants
def _mixed_cluster(seed, n_fluid=500, n_bound=300, dp=0.02):
    rng = np.random.Generator(np.random.PCG64(seed))
    rf = lattice((10, 10, 5), dp, origin=(0.5, 0.5, 0.5 + 3 * dp))
    rb = lattice((12, 12, 3), dp, origin=(0.5 - dp, 0.5 - dp, 0.5))
    rf = rf[:n_fluid] + rng.normal(0, 0.15 * dp, size=(min(n_fluid, len(rf)), 3))
    rb = rb[:n_bound]
    r = np.concatenate([rf, rb])
    n = len(r)
    t = np.concatenate([np.zeros(len(rf), np.int32), np.ones(len(rb), np.int32)])
    u = rng.normal(0, 0.3, size=(n, 3))
    u[t != 0] = 0.0
    rho = 1000.0 + rng.normal(0, 3.0, size=n)
    return oracle.State(r, u, rho, t)


def test_pair_forces_are_antisymmetric():
    # Summed over all particles the pair part of m a_i cancels (Eq. 3 with
    # grad_i W_ij = -grad_j W_ji and a symmetric Pi_ij); boundary particles sum
    # over fluid neighbours, fluid particles over all.
    dp = 0.02
    case = big_case(dp, alpha=0.1)
    st = _mixed_cluster(5)
    drho, acc, mumax, nn = oracle.derivatives(case, st)
    pair = acc.copy()
    pair[st.type == 0, 2] += case.g
    m = 1000.0 * dp ** 3
    total = m * pair.sum(axis=0)
    scale = m * np.abs(pair).sum()
    assert scale > 0
    assert np.all(np.abs(total) < 1e-12 * scale)


def test_galilean_invariance():
    dp = 0.02
    case = big_case(dp, alpha=0.1)
    rng = np.random.Generator(np.random.PCG64(9))
    r = lattice((9, 9, 9), dp) + rng.normal(0, 0.1 * dp, size=(729, 3))
    u = rng.normal(0, 0.5, size=(729, 3))
    rho = 1000.0 + rng.normal(0, 2.0, size=729)
    a = oracle.derivatives(case, fluid_state(r, rho=rho, u=u))
    b = oracle.derivatives(case, fluid_state(r, rho=rho, u=u + np.array([1.3, -0.7, 2.1])))
    for x, y in zip(a[:2], b[:2]):
        assert np.allclose(x, y, rtol=1e-9, atol=1e-9 * np.abs(x).max())


def test_viscosity_switch_linearity_and_sound_speed_readings():
    # Eqs. 4-5 on one pair of fluid particles: the viscous part of the
    # acceleration (minus that of the same pair at rest) opposes the approach
    # along the line of centres, is linear in the approach speed, vanishes for
    # a receding pair, and is proportional to c_bar, so that the EOS reading of
    # c_i (c0 (rho/rho0)^3 for gamma = 7) and the constant one (c_i = c0) differ
    # by exactly the factor (rho/rho0)^3.
    dp, rho = 0.02, 1006.0
    h = HF * dp
    ce = big_case(dp, alpha=0.1)
    cc = big_case(dp, alpha=0.1, csound_mode=1)
    r = np.array([[1.0, 1.0, 1.0], [1.0 + 1.2 * h, 1.0, 1.0]])

    def visc(case, v):
        u = np.array([[v, 0.0, 0.0], [-v, 0.0, 0.0]])
        a = oracle.derivatives(case, fluid_state(r, rho=rho, u=u))[1]
        a0 = oracle.derivatives(case, fluid_state(r, rho=rho))[1]
        return a - a0

    ve = visc(ce, 0.1)
    assert ve[0, 0] < 0.0 < ve[1, 0]
    assert np.all(ve[:, 1:] == 0.0)
    assert np.allclose(visc(ce, 0.2), 2.0 * ve, rtol=1e-12, atol=0.0)
    assert np.all(visc(ce, -0.1) == 0.0)
    assert np.allclose(ve, (rho / 1000.0) ** 3 * visc(cc, 0.1), rtol=1e-12, atol=0.0)


def test_viscosity_magnitude_matches_eq32():
    # The overall factor of Eqs. 4-5, against the viscosity the paper assigns to
    # alpha (Eq. 32: nu0 = alpha h c0 / (2 (d + 2)), d = 3).  With uniform density
    # (P = 0, c_i = c0) and a flow u = (f(x), 0, 0) with f strictly decreasing,
    # every pair with x_i != x_j approaches, so the switch is on wherever it
    # matters.  Expanding u_j - u_i to second order in the pair sum turned into
    # an integral, the first-order part cancels by symmetry and the second gives
    # a_x = (alpha c0 h / 2) f'' (-int s_x^4 F(s) / s^2 d^3s), where
    # int s_x^4 F / s^2 d^3s = (4 pi / 5) int s^3 W'(s) ds = -3/5 (integration by
    # parts and int W = 1).  So a_x = 3 nu0 f'': for f = -eps x - beta x^2 a
    # uniform -6 nu0 beta.  On a lattice with h = 1.2 sqrt(3) dp, and eta^2 =
    # 0.01 h^2 in mu, the interior value comes within 0.1 % of it.
    dp = 0.02
    h = HF * dp
    case = big_case(dp, alpha=0.1)
    r = lattice((17, 17, 17), dp)
    x = r[:, 0] - r[:, 0].mean()
    beta, eps = 1.0, 1.0  # f' = -eps - 2 beta x < 0 across the block (|x| < 0.17 m)
    u = np.zeros_like(r)
    u[:, 0] = -eps * x - beta * x * x
    acc = oracle.derivatives(case, fluid_state(r, rho=1000.0, u=u))[1]
    inner = np.all((r > r.min(axis=0) + 2 * h) & (r < r.max(axis=0) - 2 * h), axis=1)
    assert inner.sum() == 343
    nu0 = 0.1 * h * case.c0 / 10.0
    expected = -6.0 * nu0 * beta
    assert np.allclose(acc[inner, 0], expected, rtol=0.01, atol=0.0)
    assert np.max(np.abs(acc[inner, 1])) < 1e-10 * abs(expected)


def test_pressure_term_of_a_linear_pressure_field():
    # The magnitude and sign of the pressure term of Eq. 3.  With gamma = 1
    # (Eq. 8 linear, pinned above) rho = rho0 + G x / c0^2 makes P = G x exactly.
    # On a uniform lattice the pair sum becomes (rho0 / rho^2) int (P_i + P(x_i +
    # s_x)) F(s) s d^3s: the P_i part vanishes by symmetry and the linear part
    # gives G int s_x^2 F d^3s = G (4 pi / 3) int s^3 W'(s) ds = -G, so a_x =
    # -grad P / rho up to terms of order P / (rho c0^2) (below 6e-4 here).
    dp, G = 0.02, 1000.0
    h = HF * dp
    case = big_case(dp, gamma=1.0)
    r = lattice((17, 17, 17), dp)
    x = r[:, 0] - r[:, 0].mean()
    rho = 1000.0 + G * x / case.c0 ** 2
    acc = oracle.derivatives(case, fluid_state(r, rho=rho))[1]
    inner = np.all((r > r.min(axis=0) + 2 * h) & (r < r.max(axis=0) - 2 * h), axis=1)
    assert np.allclose(acc[inner, 0], -G / rho[inner], rtol=5e-3, atol=0.0)
    assert np.max(np.abs(acc[inner, 1])) < 1e-10 * G / 1000.0
    assert np.allclose(acc[inner, 2], -case.g, rtol=0.0, atol=1e-10)


def test_hydrostatic_column_balances_gravity():
    # With the hydrostatic initial density the pressure term of Eq. 3 must cancel
    # gravity inside the column (away from walls, floor and surface).
    c = wl.small_dambreak()
    case = oracle.make_case(c.tank, (1.0, 0.5, 0.3), dp=c.dp, h=c.h, c0=c.c0, alpha=c.alpha)
    st = oracle.scene(case)
    drho, acc, mumax, nn = oracle.derivatives(case, st)
    f = st.type == 0
    r = st.r
    away = f & (r[:, 0] > 3 * c.h) & (r[:, 0] < 1.0 - 3 * c.h) & (r[:, 1] > 3 * c.h) & \
        (r[:, 1] < 0.5 - 3 * c.h) & (r[:, 2] > 3 * c.h) & (r[:, 2] < 0.3 - 3 * c.h)
    assert away.sum() > 50
    # (the residual, about 2% of g at mid depth, is the discretisation error of
    # the (P_i + P_j)/(rho_i rho_j) form under a density gradient)
    assert np.max(np.abs(acc[away, 2])) < 0.05 * 9.81
    assert np.max(np.abs(acc[away, :2])) < 1e-6 * 9.81
    # Eq. 33 at depth d reproduces rho0 g d inside the column
    pts = np.array([[0.5, 0.25, z] for z in (0.08, 0.15, 0.22)])
    p = oracle.probe_pressure(case, st, pts)
    assert np.allclose(p, 1000.0 * 9.81 * (0.3 - pts[:, 2]), rtol=0.02)


# ---------------------------------------------------------------- Eq. 15
def test_dt_closed_forms():
    dp = 0.02
    case = big_case(dp, alpha=0.0)
    h = case.h
    # a lone fluid particle at rest: |f| = g and mu = 0
    st = fluid_state(np.array([[1.0, 1.0, 1.0]]))
    d = oracle.derivatives(case, st)
    assert abs(oracle.dt(case, st.type, d[3], d[1], d[2]) - 0.2 * min(math.sqrt(h / 9.81), h / case.c0)) < 1e-15
    # two fluid particles separating along x at relative speed 2v, rho = rho0
    # (no pressure, no viscosity): mu = h (2v) d / (d^2 + 0.01 h^2)
    for v, sign in [(40.0, 1.0), (40.0, -1.0)]:
        dist = 1.5 * dp
        r = np.array([[1.0, 1.0, 1.0], [1.0 + dist, 1.0, 1.0]])
        u = np.array([[-sign * v, 0, 0], [sign * v, 0, 0]], np.float64)
        st = fluid_state(r, u=u)
        d = oracle.derivatives(case, st)
        mu = h * 2 * v * dist / (dist ** 2 + 0.01 * h * h) if sign > 0 else 0.0
        expect = 0.2 * min(math.sqrt(h / 9.81), h / (case.c0 + mu))
        assert abs(oracle.dt(case, st.type, d[3], d[1], d[2]) - expect) < 1e-15 * expect / 1e-3


# ---------------------------------------------------------------- Eqs. 9-14
def test_free_fall_is_exact():
    # Constant acceleration: both the Verlet and the first-order step reproduce
    # z = z0 - g t^2 / 2 and w = -g t exactly.
    dp = 0.02
    case = big_case(dp)
    st = fluid_state(np.array([[1.0, 1.0, 1.9]]))
    dt = 1e-3
    oracle.run(case, st, 100, dt_fixed=dt)
    t = 100 * dt
    assert abs(st.r[0, 2] - (1.9 - 0.5 * 9.81 * t * t)) < 1e-12
    assert abs(st.u[0, 2] + 9.81 * t) < 1e-12
    assert abs(st.rho[0] - 1000.0) == 0.0


def test_verlet_odd_even_levels_and_resync():
    # g = 0, lone particle, u^{t-dt} = 0 and u^t = 1 entered at step 1: the
    # Verlet step u^{t+dt} = u^{t-dt} + 2 dt a alternates 0, 1, 0, ... until the
    # first-order step at step 40 copies u^40 = 0 and ends the alternation.
    dp = 0.02
    case = big_case(dp, g=0.0)
    st = oracle.State(np.array([[1.0, 1.0, 1.0]]), np.array([[1.0, 0, 0]]), np.array([1000.0]),
                      np.zeros(1, np.int32), uprev=np.zeros((1, 3)), step=1)
    dt = 1e-3
    seen = []
    for _ in range(45):
        oracle.step(case, st, dt_fixed=dt)
        seen.append(st.u[0, 0])
    # after the step with index n the velocity is u^{n+1}
    expect = [0.0 if (n + 1) % 2 == 0 else 1.0 for n in range(1, 40)] + [0.0] * 6
    assert seen == expect
    # position: x advances by dt u^n each step (a = 0)
    assert abs(st.r[0, 0] - (1.0 + dt * (1.0 + sum(expect[:-1])))) < 1e-13


def test_symplectic_free_fall_is_exact():
    # Constant acceleration: the half-step predictor and corrector reproduce
    # r = r0 + u0 t - g t^2 / 2 ez and u = u0 - g t ez exactly; a corrector that
    # advanced r with the predicted or the old velocity would not.
    case = big_case(0.02, integrator=oracle.SYMPLECTIC)
    u0 = np.array([[0.3, -0.2, 0.5]])
    st = fluid_state(np.array([[1.0, 1.0, 1.9]]), u=u0.copy())
    dt = 1e-3
    oracle.run(case, st, 100, dt_fixed=dt)
    t = 100 * dt
    expect = np.array([1.0 + 0.3 * t, 1.0 - 0.2 * t, 1.9 + 0.5 * t - 0.5 * 9.81 * t * t])
    assert np.max(np.abs(st.r[0] - expect)) < 1e-12
    assert np.max(np.abs(st.u[0] - np.array([0.3, -0.2, 0.5 - 9.81 * t]))) < 1e-12
    assert st.rho[0] == 1000.0


def _block_state(seed):
    dp = 0.02
    r = lattice(6, dp, origin=(0.8, 0.8, 0.8))
    rng = np.random.Generator(np.random.PCG64(seed))
    r = r + rng.normal(0.0, 0.05 * dp, r.shape)
    u = rng.normal(0.0, 0.05, r.shape)
    rho = 1000.0 + rng.normal(0.0, 0.5, r.shape[0])
    return fluid_state(r, rho=rho, u=u)


@pytest.mark.parametrize("integ", [oracle.SYMPLECTIC, oracle.VERLET])
def test_integrators_converge_at_second_order(integ):
    # A jittered free-standing block under pressure, gravity and the continuity
    # coupling (alpha = delta = 0 keep the right-hand side smooth), advanced to
    # the same time with dt, dt/2 and dt/4: against a dt/32 reference the
    # position error falls by ~4 per halving.  A corrector that mixed the
    # level-n and mid-step accelerations in the velocity (u' + dt/2 Du') would
    # fall by ~2 only.
    dt0, n0 = 4e-4, 10
    case = big_case(0.02, alpha=0.0, delta=0.0, ns=10 ** 6, integrator=integ)

    def final(k):
        st = _block_state(3)
        oracle.run(case, st, n0 * k, dt_fixed=dt0 / k)
        return st.r

    ref = final(32)
    err = [np.max(np.abs(final(k) - ref)) for k in (1, 2, 4)]
    rates = [err[0] / err[1], err[1] / err[2]]
    assert all(3.3 < q < 4.8 for q in rates), (err, rates)


def test_symplectic_density_rises_under_compression():
    # u = -eps (r - c): D rho/Dt = 3 eps rho0 in the interior; one symplectic
    # step of dt raises the central density by 3 eps rho0 dt to first order
    # (sign and factor of the (2 - e)/(2 + e) update).
    dp = 0.02
    case = big_case(dp, delta=0.0, g=0.0, integrator=oracle.SYMPLECTIC)
    r = lattice(13, dp)
    c = r.mean(axis=0)
    eps = 0.5
    st = fluid_state(r, u=-eps * (r - c))
    centre = np.argmin(np.linalg.norm(r - c, axis=1))
    dt = 1e-4
    oracle.step(case, st, dt_fixed=dt)
    gain = st.rho[centre] - 1000.0
    assert gain > 0
    assert abs(gain / (3 * eps * 1000.0 * dt) - 1.0) < 0.03


@pytest.mark.parametrize("integ", [oracle.VERLET, oracle.SYMPLECTIC])
def test_gate_moves_at_its_prescribed_velocity(integ):
    # Gate particles (Section 3.2: a gate lifted at constant speed) follow
    # r = r0 + v t exactly and keep u = v, whatever the fluid does to them.
    c = wl.small_gate_dambreak()
    case = oracle.make_case(c.tank, c.column, dp=0.04, h=HF * 0.04, c0=c.c0, gate=c.gate,
                            gate_velocity=c.gate_velocity, integrator=integ)
    st = oracle.scene(case)
    gate = st.type == oracle.GATE
    assert gate.sum() == 1 * 13 * 13  # one lattice layer of 0.04 m, 0.5 x 0.5 m
    r0 = st.r[gate].copy()
    dt = 2e-4
    oracle.run(case, st, 20, dt_fixed=dt)
    t = 20 * dt
    assert np.max(np.abs(st.r[gate] - (r0 + np.array(c.gate_velocity) * t))) < 1e-13
    assert np.all(st.u[gate] == np.array(c.gate_velocity))


def test_continuity_sees_the_gate_velocity():
    # A fluid block and a gate moving together at the same velocity, uniform
    # density, no gravity: every relative velocity is zero, so Eq. 7 gives
    # D rho/Dt = 0 for every fluid and gate particle.  The same block against a
    # gate at rest compresses next to it.
    dp = 0.02
    case = big_case(dp, g=0.0, delta=0.0)
    fluid = lattice((6, 6, 6), dp, origin=(0.8, 0.8, 0.8))
    gate = lattice((2, 6, 6), dp, origin=(0.8 + 6 * dp, 0.8, 0.8))
    r = np.concatenate([fluid, gate])
    t = np.concatenate([np.zeros(len(fluid), np.int32), np.full(len(gate), oracle.GATE, np.int32)])
    v = np.array([0.3, 0.0, 0.7])
    for gate_v, moving_together in ((v, True), (np.zeros(3), False)):
        u = np.concatenate([np.tile(v, (len(fluid), 1)), np.tile(gate_v, (len(gate), 1))])
        st = oracle.State(r, u, np.full(len(r), 1000.0), t)
        drho, acc, mumax, nn = oracle.derivatives(case, st)
        if moving_together:
            assert np.max(np.abs(drho)) < 1e-9
        else:
            # the fluid moving into the resting gate (v_x > 0) raises its density
            assert drho[:len(fluid)].max() > 1.0 and drho[len(fluid):].max() > 1.0


# ---------------------------------------------------------------- probes and diagnostics
def test_shepard_probe_of_uniform_density_is_the_eos_value():
    c = wl.tiny_case()
    case = oracle.make_case(c.tank, c.column, dp=c.dp, h=c.h, c0=c.c0, init_mode=1)
    st = oracle.scene(case)
    st.rho[:] = 1004.0
    p = oracle.probe_pressure(case, st, np.array([[0.1, 0.2, 0.05], [0.25, 0.1, 0.15], [0.9, 0.2, 0.3]]))
    expect = oracle.tait(case, 1004.0)
    assert abs(p[0] - expect) < 1e-9 * expect and abs(p[1] - expect) < 1e-9 * expect
    assert p[2] == 0.0  # no fluid within 2h


def test_wave_height_of_still_column():
    c = wl.tiny_case(0.02)
    case = oracle.make_case(c.tank, c.column, dp=c.dp, h=c.h, c0=c.c0)
    st = oracle.scene(case)
    hgt = oracle.probe_wave_height(case, st, np.array([[0.15, 0.2], [0.7, 0.2]]))
    assert abs(hgt[0] - 0.2) <= 0.5 * c.dp
    assert hgt[1] == 0.0


def test_force_on_submerged_box_at_rest():
    # A box on the floor under a hydrostatic column: horizontal face loads cancel
    # by symmetry and the vertical load is the weight of water above it,
    # rho0 g (H - hb) A (no fluid under the box).  The boundary particles carry
    # the hydrostatic density they reach once the dynamic boundary has relaxed.
    dp = 0.02
    H = 0.3
    hb = 0.1
    box = (0.4, 0.1, 0.0, 0.2, 0.2, hb)
    c0 = 10 * math.sqrt(9.81 * H)
    case = oracle.make_case((1.0, 0.4, 0.4), (1.0, 0.4, H), box, dp=dp, h=HF * dp, c0=c0)
    st = oracle.scene(case)
    inside = np.all((st.r >= np.array(box[:3])) & (st.r <= np.array(box[:3]) + np.array(box[3:])), axis=1)
    keep = ~((st.type == 0) & inside)
    st = oracle.State(st.r[keep], st.u[keep], st.rho[keep], st.type[keep])
    depth = np.maximum(H - st.r[:, 2], 0.0)
    st.rho[:] = 1000.0 * (1.0 + 7.0 * 9.81 * depth / c0 ** 2) ** (1.0 / 7.0)
    f = oracle.probe_force(case, st)
    load = 1000.0 * 9.81 * (H - hb) * box[3] * box[4]
    assert abs(f[0]) < 1e-9 * load and abs(f[1]) < 1e-9 * load
    assert f[2] < 0 and abs(-f[2] / load - 1.0) < 0.05


def test_diagnostics_of_still_column():
    c = wl.tiny_case()
    case = oracle.make_case(c.tank, c.column, dp=c.dp, h=c.h, c0=c.c0, init_mode=1)
    st = oracle.scene(case)
    d = oracle.diagnostics(case, st)
    m = 1000.0 * c.dp ** 3
    nf = int((st.type == 0).sum())
    assert abs(d[0] - m * st.n) < 1e-9 * m * st.n
    assert abs(d[1] - nf * c.dp ** 3) < 1e-12
    assert np.all(d[2:6] == 0.0) and d[7] == 0.0 and d[8] == 0.0 and d[9] == nf
    # potential energy: layers k = 0 .. nz-1 at z = (k + 1/2) dp
    nz = int(round(c.column[2] / c.dp))
    per_layer = nf // nz
    epot = m * 9.81 * per_layer * sum((k + 0.5) * c.dp for k in range(nz))
    assert abs(d[6] - epot) < 1e-9 * epot


def test_scene_counts_match_lattice_layout():
    for c in (wl.small_dambreak(), wl.obstacle_dambreak(), wl.tiny_case(obstacle=True)):
        case = oracle.make_case(c.tank, c.column, c.obstacle, dp=c.dp, h=c.h, c0=c.c0)
        assert tuple(oracle.scene_counts(case)) == c.lattice_counts()
    assert wl.small_dambreak().lattice_counts() == (7500, 11032, 0)


def test_internal_energy_is_the_integral_of_p_over_rho_squared():
    # Diagnostics slot 7 is sum m e(rho) with de/drho = P/rho^2 (Eq. 8) and
    # e(rho0) = 0: pinned by quadrature of P/rho^2 and by its derivative.
    c = wl.tiny_case()
    case = oracle.make_case(c.tank, c.column, dp=c.dp, h=c.h, c0=c.c0, init_mode=1)
    m = 1000.0 * c.dp ** 3

    def energy(rho):
        st = oracle.State(np.array([[0.1, 0.1, 0.1]]), np.zeros((1, 3)), np.array([rho]), np.zeros(1, np.int32))
        return oracle.diagnostics(case, st)[7]

    assert energy(1000.0) == 0.0
    for rho in (940.0, 990.0, 1003.0, 1030.0, 1100.0):
        quad, _ = integrate.quad(lambda s: oracle.tait(case, s) / s ** 2, 1000.0, rho, epsabs=1e-13, epsrel=1e-12)
        assert abs(energy(rho) - m * quad) <= 1e-9 * abs(m * quad)
        d = 1e-3
        fd = (energy(rho + d) - energy(rho - d)) / (2 * d)
        expect = m * oracle.tait(case, rho) / rho ** 2
        assert abs(fd - expect) <= 1e-6 * abs(expect)


def test_momentum_and_kinetic_energy_of_a_moving_state():
    # Diagnostics slots 2-5 on non-zero velocities: sum m u and sum m |u|^2 / 2
    # over the fluid particles (boundary particles carry none).
    c = wl.tiny_case()
    case = oracle.make_case(c.tank, c.column, dp=c.dp, h=c.h, c0=c.c0, init_mode=1)
    st = oracle.scene(case)
    rng = np.random.Generator(np.random.PCG64(11))
    f = st.type == 0
    st.u[f] = rng.normal(0.0, 1.5, (int(f.sum()), 3)) + np.array([0.4, -0.2, 0.1])
    d = oracle.diagnostics(case, st)
    m = 1000.0 * c.dp ** 3
    mom = m * st.u[f].sum(axis=0)
    ke = 0.5 * m * float((st.u[f] ** 2).sum())
    assert np.allclose(d[2:5], mom, rtol=1e-12, atol=1e-12 * m)
    assert abs(d[5] - ke) <= 1e-12 * ke
    st.u[~f] = 5.0  # boundary velocities do not enter
    assert np.array_equal(oracle.diagnostics(case, st)[2:6], d[2:6])


# ---------------------------------------------------------------- delta term near boundaries
def test_delta_mode_full_support_drops_the_term_next_to_boundaries():
    # A fluid block at rest on two layers of floor particles, its density
    # growing linearly with depth.  With u = 0 only the delta term of Eq. 7 is
    # left.  DELTA_ALL_FLUID: next to the floor the fluid-only sum is one-sided
    # and drains density.  DELTA_FULL_SUPPORT: every fluid particle with a floor
    # particle within 2h has a rate of exactly zero; all others keep the rate of
    # the first mode.
    dp = 0.02
    h = HF * dp
    fluid = lattice((12, 12, 10), dp)
    floor = lattice((12, 12, 2), dp, origin=(0.5, 0.5, 0.5 - 2 * dp))
    r = np.vstack([fluid, floor])
    ztop = fluid[:, 2].max()
    rho = 1000.0 + 5.0 * (ztop - r[:, 2]) / dp
    typ = np.r_[np.zeros(len(fluid), np.int32), np.ones(len(floor), np.int32)]
    st = oracle.State(r, np.zeros_like(r), rho, typ)
    d_all = oracle.derivatives(big_case(dp, delta_mode=oracle.DELTA_ALL_FLUID), st)[0]
    d_full = oracle.derivatives(big_case(dp, delta_mode=oracle.DELTA_FULL_SUPPORT), st)[0]
    dist = np.sqrt(((fluid[:, None, :] - floor[None, :, :]) ** 2).sum(axis=2)).min(axis=1)
    near = np.r_[dist < 2 * h, np.zeros(len(floor), bool)]
    f = typ == 0
    assert near.sum() > 100 and (f & ~near).sum() > 100
    assert np.all(d_full[near] == 0.0)
    assert np.array_equal(d_full[f & ~near], d_all[f & ~near])
    bottom = f & (r[:, 2] < fluid[:, 2].min() + 0.5 * dp) & np.all(np.abs(r[:, :2] - fluid[:, :2].mean(axis=0)) < 2 * dp, axis=1)
    assert bottom.sum() >= 4 and np.all(d_all[bottom] < 0.0)


def _still_column(delta, integrator, delta_mode, t_end=1.5):
    """A column covering the floor of a 0.18 x 0.18 m tank, 0.4 m deep, started
    at uniform density with alpha = 0.1.  Returns, at points from 2h above the
    floor to 4h below the surface (away from both truncated supports): the
    Eq. 33 pressure over rho0 g d, d measured from the height z0 where the
    fitted linear pressure profile vanishes; the fitted vertical gradient over
    -rho0 g; and z0 minus the particle surface (top fluid layer + dp/2)."""
    dp, H, L = 0.02, 0.4, 0.18
    case = oracle.make_case((L, L, H + 0.1), (L, L, H), dp=dp, h=HF * dp, c0=10.0 * math.sqrt(9.81 * H),
                            alpha=0.1, delta=delta, init_mode=1, cell_div=1, integrator=integrator,
                            delta_mode=delta_mode)
    st = oracle.scene(case)
    threads = oracle.set_threads(os.cpu_count() or 1)
    t = 0.0
    while t < t_end:
        t += oracle.run(case, st, 50).sum()
    oracle.set_threads(threads)
    zf = st.r[st.type == 0, 2]
    zs = zf[zf > zf.max() - 0.5 * dp].mean() + 0.5 * dp
    pts = np.array([[L / 2, L / 2, z] for z in np.arange(2 * case.h, zs - 4 * case.h, dp)])
    p = oracle.probe_pressure(case, st, pts)
    a, b = np.polyfit(pts[:, 2], p, 1)
    z0 = -b / a
    return p / (1000.0 * 9.81 * (z0 - pts[:, 2])), a / (-1000.0 * 9.81), z0 - zs


def test_still_column_relaxes_to_hydrostatic_pressure():
    # The check the method must pass: a still column settles to P = rho0 g d
    # (Eq. 8 with the momentum balance of Eq. 3) within 2 % away from the walls,
    # with the free surface (P = 0) within dp/2 of the particle surface; here
    # with the paper's integrator (Eqs. 9-14) and the delta term off.
    ratio, slope, dz = _still_column(0.0, oracle.VERLET, oracle.DELTA_ALL_FLUID)
    assert len(ratio) >= 6
    assert np.all(np.abs(ratio - 1.0) <= 0.02), ratio
    assert abs(slope - 1.0) <= 0.02, slope
    assert abs(dz) <= 0.5 * 0.02, dz


def test_still_column_with_delta_over_full_supports():
    # With delta = 0.1 the delta term over fluid neighbours only is one-sided
    # next to the floor and drains the deep density (about 12 % low after 1.5 s,
    # not asserted); with the term dropped next to boundaries the column holds
    # the hydrostatic pressure like the column without the term.
    ratio, slope, dz = _still_column(0.1, oracle.SYMPLECTIC, oracle.DELTA_FULL_SUPPORT, t_end=1.0)
    assert np.all(np.abs(ratio - 1.0) <= 0.02), ratio
    assert abs(slope - 1.0) <= 0.02, slope
    assert abs(dz) <= 0.5 * 0.02, dz

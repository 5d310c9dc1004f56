"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against what the paper prints, against a closed
form, a textbook formula, an invariant, or brute force, chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import temperature_noise, uniform01

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------------------
# textbook equilibria and Guo forcing (independent of the printed moments)
# ---------------------------------------------------------------------------


def _textbook_weights(lat):
    """Standard lattice weights by speed class (Qian, d'Humieres & Lallemand 1992)."""
    sq = (lat.e ** 2).sum(axis=1)
    if lat.q == 9:
        table = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    else:
        table = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}
    return np.array([table[int(s)] for s in sq])


def _hermite_feq(lat, rho, u):
    w = _textbook_weights(lat)
    eu = lat.e @ u
    usq = float(u @ u)
    return w * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * usq)


def _guo_force(lat, u, F):
    """Guo, Zheng & Shi (2002): F~_i = w_i [3 e.F + 9 (e.u)(e.F) - 3 u.F]."""
    w = _textbook_weights(lat)
    eu = lat.e @ u
    eF = lat.e @ F
    return w * (3 * eF + 9 * eu * eF - 3 * float(u @ F))


def _rand(n, seed, lo=-1.0, hi=1.0):
    return lo + (hi - lo) * uniform01(n, seed)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19], ids=lambda l: l.name)
def test_printed_equilibrium_moments_match_hermite_equilibrium(lat):
    for seed in range(5):
        r = _rand(lat.d + 1, seed)
        rho = 1.0 + 0.1 * r[0]
        u = 0.1 * r[1:]
        m_printed = np.array(lat.meq(rho, list(u)), dtype=float)
        m_textbook = lat.M @ _hermite_feq(lat, rho, u)
        np.testing.assert_allclose(m_textbook, m_printed, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19], ids=lambda l: l.name)
def test_printed_forcing_moments_match_guo(lat):
    for seed in range(5):
        r = _rand(2 * lat.d, 100 + seed)
        u, F = 0.1 * r[:lat.d], 1e-3 * r[lat.d:]
        m_printed = np.array(lat.mforce(list(u), list(F)), dtype=float)
        m_textbook = lat.M @ _guo_force(lat, u, F)
        np.testing.assert_allclose(m_textbook, m_printed, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", [O.D2Q5, O.D3Q7], ids=lambda l: l.name)
def test_thermal_equilibrium_moments_and_anti_bounce_back_weight(lat):
    """sum g^eq = T, sum e g^eq = u T, second moment = c_sT^2 T with c_sT^2 = omega
    (the printed anti-bounce-back weight is twice the rest-frame equilibrium weight)."""
    a_T = -3.5
    T, u = 0.37, np.array([0.05, -0.03, 0.02][:lat.d])
    geq = lat.Ninv @ np.array(lat.neq(T, list(u), a_T), dtype=float)
    assert abs(geq.sum() - T) < 1e-15
    np.testing.assert_allclose(lat.e.T @ geq, u * T, atol=1e-15)
    g0 = lat.Ninv @ np.array(lat.neq(1.0, [0.0] * lat.d, a_T), dtype=float)
    for i in range(1, lat.q):
        assert abs(2 * g0[i] - lat.omega(a_T)) < 1e-15
    # isotropic second moment: c_sT^2 equals omega on every axis
    for a in range(lat.d):
        assert abs((lat.e[:, a] ** 2) @ g0 - lat.omega(a_T)) < 1e-15


@pytest.mark.parametrize("lat", [O.D2Q5, O.D3Q7], ids=lambda l: l.name)
def test_a_T_formula_implies_q_j(lat):
    """alpha = c_sT^2 (1/q_j - 1/2) reproduces the printed a_T(alpha) only with
    q_j = 3 - sqrt(3) (reading R4)."""
    q_j = 3 - math.sqrt(3)
    for alpha in (1e-3, 0.01, 0.05, 0.14):
        a_T = lat.a_T_of_alpha(alpha)
        assert abs(lat.omega(a_T) * (1 / q_j - 0.5) - alpha) < 1e-15


# ---------------------------------------------------------------------------
# collision invariants
# ---------------------------------------------------------------------------


def _small_cavity(d=2, n=6, **kw):
    xi = O.mesh_erf(n, 1.5)
    p = O.Params(Ra=kw.pop("Ra", 1e5), **kw)
    return O.Cavity(xi, xi, xi if d == 3 else None, params=p)


@pytest.mark.parametrize("d", [2, 3])
def test_collision_conserves_mass_and_adds_exactly_F(d):
    cav = _small_cavity(d)
    shape = cav.shape
    rng_f = 1.0 / cav.flow.q * (1 + 0.05 * _rand(cav.flow.q * int(np.prod(shape)), 7)).reshape(
        (cav.flow.q,) + shape)
    g = 0.1 * _rand(cav.thermal.q * int(np.prod(shape)), 8).reshape((cav.thermal.q,) + shape)
    rho, u, theta, F = cav.macroscopic(rng_f, g)
    fp, gp = cav.collide(rng_f, g)
    np.testing.assert_allclose(fp.sum(0), rho, atol=1e-15)
    np.testing.assert_allclose(gp.sum(0), theta, atol=1e-15)
    for a in range(d):
        ea = cav.flow.e[:, a].astype(float)
        np.testing.assert_allclose(np.tensordot(ea, fp - rng_f, axes=1), F[a], atol=2e-15)
        assert np.abs(F[1]).max() > 1e-6
    # s_rho and s_j do not change the post-collision state
    cav2 = _small_cavity(d, s_rho=0.7, s_j=1.3)
    fp2, _ = cav2.collide(rng_f, g)
    np.testing.assert_allclose(fp2, fp, atol=1e-15)


def test_equilibrium_without_force_is_a_collision_fixed_point():
    cav = _small_cavity(2, T_hot=0.0, T_cold=0.0)
    rho = 1 + 0.01 * _rand(36, 3).reshape(cav.shape)
    u = [0.02 * _rand(36, 4).reshape(cav.shape), 0.02 * _rand(36, 5).reshape(cav.shape)]
    f, g = cav.equilibrium(rho, u, np.zeros(cav.shape))
    fp, gp = cav.collide(f, g)
    np.testing.assert_allclose(fp, f, atol=1e-15)
    np.testing.assert_allclose(gp, g, atol=1e-16)


# ---------------------------------------------------------------------------
# meshes and interpolation
# ---------------------------------------------------------------------------


def test_mesh_quality_matches_paper():
    ref = json.load(open(os.path.join(GOLDEN, "mesh_quality.json")))
    growth, aspect = O.mesh_quality(O.mesh_erf(ref["N"], ref["a"]))
    assert abs(growth - ref["growth"]) < 5e-5
    assert abs(aspect - ref["aspect"]) < 5e-3


@pytest.mark.parametrize("N", [16, 63, 64, 257])
def test_length_scales_table1(N):
    xi = O.mesh_erf(N, 1.5)
    X = O.lattice_coordinates(xi)
    assert X[0] == 0 and abs(X[1] - 1) < 1e-15                     # 1 l.u. = y_1
    assert abs(O.characteristic_length(X) - (1 / xi[1] - 1)) < 1e-9  # (1/y_1 - 1) l.u.
    assert abs(O.cell_widths(X).sum() - O.characteristic_length(X)) < 1e-9
    np.testing.assert_allclose(xi + xi[::-1], 1.0, atol=1e-15)
    assert np.diff(X)[1:-1].min() > 1.0                             # spacing grows from the wall
    Xu = O.lattice_coordinates(O.mesh_uniform(N))
    assert O.characteristic_length(Xu) == N                         # N l.u.
    np.testing.assert_array_equal(O.cell_widths(Xu), np.ones(N))


def _random_mesh(N, seed):
    steps = 1.0 + 2.0 * uniform01(N + 1, seed)
    steps[0] = steps[-1] = 1.0
    return np.concatenate([[0.0], np.cumsum(steps)])


@pytest.mark.parametrize("stencil", ["centred", "upwind"])
def test_interpolation_exact_on_quadratics(stencil):
    for seed in range(4):
        X = _random_mesh(12, seed)
        a, b, c2 = _rand(3, 50 + seed)
        P = lambda x: a + b * x + c2 * x * x
        vals = P(X[1:-1])
        for c in (+1, -1):
            tab = O.interpolation_table(X, c, stencil)
            out = O.interpolate_axis(vals[None, :], 1, tab)[0]
            j = np.where(~tab.wall)[0]
            np.testing.assert_allclose(out[j], P(X[1:-1][j] - c), rtol=0, atol=1e-12)
            np.testing.assert_allclose(tab.w[j].sum(axis=1), 1.0, atol=1e-14)
            assert tab.wall.sum() == 1
            assert tab.wall[0 if c == +1 else -1]


def test_interpolation_matches_brute_force_polyfit():
    X = _random_mesh(5, 9)
    vals = _rand(5, 10)
    for c in (+1, -1):
        tab = O.interpolation_table(X, c)
        out = O.interpolate_axis(vals[None, :], 1, tab)[0]
        for j in np.where(~tab.wall)[0]:
            b = tab.base[j]
            coef = np.polyfit(X[1 + b:4 + b], vals[b:b + 3], 2)
            assert abs(np.polyval(coef, X[1 + j] - c) - out[j]) < 1e-12
            # the departure point lies between the two nearest stencil nodes
            assert X[1 + b] <= X[1 + j] - c <= X[3 + b]


def test_interpolation_is_a_pure_shift_on_the_uniform_mesh():
    X = O.lattice_coordinates(O.mesh_uniform(10))
    vals = _rand(10, 11)
    for c in (+1, -1):
        tab = O.interpolation_table(X, c)
        out = O.interpolate_axis(vals[None, :], 1, tab)[0]
        j = np.where(~tab.wall)[0]
        np.testing.assert_array_equal(out[j], vals[j - c])
        assert set(np.unique(tab.w[j])) <= {0.0, 1.0}


# ---------------------------------------------------------------------------
# wall derivative and averages
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("mesh", ["erf", "uniform"])
def test_wall_derivative_exact_on_quadratics(mesh):
    N = 20
    xi = O.mesh_erf(N, 2.1) if mesh == "erf" else O.mesh_uniform(N)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e6, T_hot=0.3, T_cold=-0.2))
    X = cav.X[0]
    for side, Tw, Xw in (("hot", 0.3, X[1] - 0.5), ("cold", -0.2, X[-2] + 0.5)):
        beta, gamma = 0.013, -0.0021
        P = Tw + beta * (X[1:-1] - Xw) + gamma * (X[1:-1] - Xw) ** 2
        T = np.broadcast_to(P, cav.shape)
        np.testing.assert_allclose(cav.wall_derivative(T, side), beta, atol=1e-14)


def test_eq16_is_the_three_point_one_sided_formula():
    """At q = 1 Eq. (17) is the textbook one-sided derivative through the wall value
    and the nodes at h/2 and 3h/2: (-8 phi_w + 9 phi_1 - phi_2)/(3h)."""
    xi = O.mesh_uniform(8)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e6, T_hot=0.25))
    T = np.zeros(cav.shape)
    T[:, 0], T[:, 1] = 0.7, -0.4
    expect = (-8 * 0.25 + 9 * 0.7 - (-0.4)) / 3
    np.testing.assert_allclose(cav.wall_derivative(T, "hot"), expect, atol=1e-15)


# ---------------------------------------------------------------------------
# whole-solver pins
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("d", [2, 3])
def test_isothermal_rest_state_is_a_fixed_point(d):
    cav = _small_cavity(d, n=8, T_hot=0.0, T_cold=0.0)
    cav.init_fields(np.zeros(cav.shape))
    f0, g0 = cav.f.copy(), cav.g.copy()
    cav.step(10)
    # unchanged to the rounding of ten steps (the weights sum to 1 only to rounding)
    np.testing.assert_allclose(cav.f, f0, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(cav.g, g0)


@pytest.mark.parametrize("mesh", ["uniform", "erf"])
def test_steady_conduction_is_linear_with_unit_nusselt(mesh):
    """Ra = 1e-6: the steady temperature is linear between the walls (the scheme is
    exact for linear fields; the buoyant flow distorts it by ~1e-10) and
    Nu_hot = Nu_cold = Nu_middle = 1."""
    N = 12
    xi = O.mesh_uniform(N) if mesh == "uniform" else O.mesh_erf(N, 1.5)
    L = O.characteristic_length(O.lattice_coordinates(xi))
    Pr, Ra, alpha = 0.71, 1e-6, 0.14
    Ma = alpha * math.sqrt(Pr * Ra) / L * math.sqrt(3)     # gives alpha = 0.14
    cav = O.Cavity(xi, xi, params=O.Params(Ra=Ra, Pr=Pr, Ma=Ma))
    assert abs(cav.par.alpha - alpha) < 1e-12
    cav.init_fields(np.zeros(cav.shape))
    cav.step(3000)
    rho, u, T = cav.fields()
    X = cav.X[0][1:-1]
    T_lin = 0.5 - (X - (cav.X[0][1] - 0.5)) / L
    np.testing.assert_allclose(T, np.broadcast_to(T_lin, T.shape), atol=1e-8)
    r = cav.reductions()
    for k in ("Nu_hot", "Nu_cold", "Nu_middle", "Nu"):
        assert abs(r[k] - 1.0) < 1e-8, (k, r[k])


def test_conduction_decay_rate_gives_the_thermal_diffusivity():
    """Transient conduction between the isothermal walls from T = 0: the deviation
    from the linear profile is odd about the centre, so its slowest mode is
    sin(2 pi x/L), which decays as exp(-alpha (2 pi/L)^2 t)."""
    Nx, Ny = 32, 4
    xi_x, xi_y = O.mesh_uniform(Nx), O.mesh_uniform(Ny)
    Ly = Ny
    Pr, Ra, alpha = 0.71, 1e-2, 0.1
    Ma = alpha * math.sqrt(Pr * Ra) / Ly * math.sqrt(3)
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=Ra, Pr=Pr, Ma=Ma))
    cav.init_fields(np.zeros(cav.shape))
    X = cav.X[0][1:-1] - 0.5                     # distance from the hot wall
    mode = np.sin(2 * np.pi * X / Nx)
    T_lin = 0.5 - X / Nx
    amps, times = [], []
    for k in range(12):
        cav.step(100)
        T = cav.fields()[2][Ny // 2]
        amps.append(((T - T_lin) @ mode) / (mode @ mode))
        times.append(cav.time)
    rate = -np.polyfit(times[3:], np.log(np.abs(amps[3:])), 1)[0]
    expect = cav.par.alpha * (2 * np.pi / Nx) ** 2
    assert abs(rate / expect - 1) < 0.01, (rate, expect)


@pytest.mark.parametrize("mesh", ["uniform", "erf"])
def test_shear_wave_decay_gives_the_viscosity(mesh):
    """v(x) = V sin(2 pi x / L_x) between the no-slip x-walls (zero net flux) in a tall
    cavity decays as exp(-nu (2 pi/L_x)^2 t) at mid-height until the sound waves
    launched by the end walls arrive (64 l.u. at c_s: ~110 steps).  A wall
    misplaced by half a lattice unit changes the rate by about 6%."""
    Nx, Ny = 32, 128
    xi_x = O.mesh_uniform(Nx) if mesh == "uniform" else O.mesh_erf(Nx, 1.0)
    xi_y = O.mesh_uniform(Ny)
    nu = 0.1
    Pr, L = 0.71, Ny
    u_f = 0.1 / math.sqrt(3)
    Ra = Pr * (u_f * L / nu) ** 2
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=Ra, Pr=Pr, T_hot=0.0, T_cold=0.0))
    assert abs(cav.par.nu - nu) < 1e-12
    Xx = cav.X[0]
    Lx = O.characteristic_length(Xx)
    xw = Xx[1:-1] - (Xx[1] - 0.5)
    mode = np.sin(2 * np.pi * xw / Lx)
    V = 1e-3
    v0 = np.broadcast_to(V * mode, cav.shape).copy()
    cav.init_fields(np.zeros(cav.shape), u=[np.zeros(cav.shape), v0])
    Wx = cav.W[0]
    amps, times = [], []
    for k in range(9):
        cav.step(10)
        v = cav.fields()[1][1][Ny // 2]
        amps.append((Wx * v * mode).sum() / (Wx * mode * mode).sum())
        times.append(cav.time)
    rate = -np.polyfit(times[1:], np.log(amps[1:]), 1)[0]
    expect = nu * (2 * np.pi / Lx) ** 2
    # the interpolation on the stretched mesh adds a little numerical viscosity
    tol = 0.01 if mesh == "uniform" else 0.02
    assert abs(rate / expect - 1) < tol, (rate, expect)


@pytest.mark.parametrize("d", [2, 3])
def test_centro_symmetry_of_the_noise_free_cavity(d):
    """With the reference temperature at the mean of the walls, rotating the cavity
    by 180 degrees about the z axis while swapping hot and cold maps the problem
    to itself: T -> -T, (u, v) -> -(u, v) at the rotated node."""
    n = 14 if d == 2 else 8
    cav = _small_cavity(d, n=n, Ra=1e6, T0=0.0)     # reference at the mean wall temperature
    cav.init_fields(np.zeros(cav.shape))
    cav.step(150)
    rho, u, T = cav.fields()
    rot = (slice(None, None, -1),) * 2 if d == 2 else (slice(None), slice(None, None, -1),
                                                      slice(None, None, -1))
    scale = np.abs(T).max()
    assert scale > 1e-3
    np.testing.assert_allclose(T + T[rot], 0, atol=1e-13 * scale + 1e-16)
    np.testing.assert_allclose(rho - rho[rot], 0, atol=1e-14)
    for a in range(2):
        np.testing.assert_allclose(u[a] + u[a][rot], 0, atol=1e-10 * np.abs(u[a]).max() + 1e-18)
    if d == 3:   # mirror symmetry in z
        np.testing.assert_allclose(T - T[::-1], 0, atol=1e-13 * scale)
        np.testing.assert_allclose(u[2] + u[2][::-1], 0, atol=1e-10 * np.abs(u[2]).max() + 1e-18)


def test_hot_wall_on_the_left_turns_the_cell_clockwise():
    """(After the early hydrostatic transient of the cold-wall reference.)"""
    cav = _small_cavity(2, n=16, Ra=1e6)
    cav.init_fields(np.zeros(cav.shape))
    cav.step(800)
    rho, u, T = cav.fields()
    mid = cav.shape[0] // 2
    assert u[1][mid, 1] > 0 and u[1][mid, -2] < 0       # rises at the hot wall
    assert u[0][-2, cav.shape[1] // 2] > 0              # moves right along the top
    assert T[mid, 0] > 0 > T[mid, -1]


def test_mass_drift_is_bounded():
    xi = O.mesh_tanh(32, 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e6))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    m0 = cav.reductions()["mass"]
    cav.step(1000)
    assert abs(cav.reductions()["mass"] / m0 - 1) < 1e-6


# ---------------------------------------------------------------------------
# convergence arithmetic against the paper's tables
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("name", ["table2_ra1e6.json", "table2_ra1e8.json"])
def test_richardson_and_gci_reproduce_table2(name):
    ref = json.load(open(os.path.join(GOLDEN, name)))
    for key in ("Nu", "Nu_hot", "Nu_middle", "Re"):
        row = ref[key]
        Fc, Fm, Ff = row["values"]
        p, Finf = O.richardson(Fc, Fm, Ff, 2.0)
        # the table inputs are rounded to 4 decimals, so p carries their rounding error
        dp = 0.5e-4 * (abs(1 / (Fc - Fm)) + 2 * abs(1 / (Fm - Ff))) / math.log(2) * 2
        assert abs(p - row["p"]) < 0.05 + dp, (key, p)
        assert abs(Finf - row["inf"]) < 2e-4 * max(1, abs(row["inf"]) / 10), (key, Finf)
        g = O.gci_fine(Fm, Ff, row["p"], 2.0)
        assert abs(g / row["gci_percent"] - 1) < 0.2, (key, g)


def test_table3_local_orders():
    """u_c and v_c carry five significant digits, enough to reproduce the printed
    orders (T_c is printed to 5 decimals, so its differences are rounding)."""
    ref = json.load(open(os.path.join(GOLDEN, "table3_ra1e6.json")))
    for key in ("u_c", "v_c"):
        p, Finf = O.richardson(*ref[key]["values"], 2.0)
        assert abs(p - ref[key]["p"]) < 0.1, (key, p)
        assert abs(Finf / ref[key]["inf"] - 1) < 3e-3, (key, Finf)


# ---------------------------------------------------------------------------
# the steady criterion and the volume reductions on states with closed forms
# ---------------------------------------------------------------------------


def test_steady_change_closed_forms():
    rng = np.random.default_rng(5)
    u = [rng.standard_normal((6, 7)), rng.standard_normal((6, 7))]
    T = rng.uniform(0.1, 0.9, (6, 7))
    assert O.steady_change(u, u, T, T) == (0.0, 0.0)
    # doubling every velocity changes each node by its own speed: du = 1
    du, dT = O.steady_change([2 * c for c in u], u, T, T)
    assert abs(du - 1.0) < 1e-15 and dT == 0.0
    # a uniform shift c of T*: dT = c N / sum |T*|
    du, dT = O.steady_change(u, u, T + 0.01, T)
    assert abs(dT - 0.01 * T.size / np.abs(T).sum()) < 1e-15


@pytest.mark.parametrize("mesh", ["uniform", "erf"])
def test_volume_reductions_of_uniform_and_two_valued_flows(mesh):
    """T* uniform and a uniform or half-and-half horizontal velocity: <Nu>,
    the RMS <Re> (R10) and the mean-speed Re_mean have closed forms (the mesh is
    symmetric, so each half of the columns carries half the volume)."""
    n = 16
    xi = O.mesh_uniform(n) if mesh == "uniform" else O.mesh_erf(n, 1.5)
    p = O.Params(Ra=1e6, Pr=0.71)
    cav = O.Cavity(xi, xi, params=p)
    uf = cav.par.u_f
    Tstar = 0.3                              # T* = (T - T_cold) / dT
    T = np.full(cav.shape, p.T_cold + Tstar * (p.T_hot - p.T_cold))
    c1, c2 = 0.02 * uf, -0.05 * uf
    # uniform velocity
    cav.init_fields(T, [np.full(cav.shape, c1), np.zeros(cav.shape)])
    r = cav.reductions()
    assert abs(r["Nu"] - (math.sqrt(p.Ra * p.Pr) * (c1 / uf) * Tstar + 1.0)) < 1e-12
    # the buoyancy force of T* = 0.3 shifts the reported v by F / 2 rho; use T* = 0 for Re
    T0 = np.full(cav.shape, p.T_cold)
    cav.init_fields(T0, [np.full(cav.shape, c1), np.zeros(cav.shape)])
    r = cav.reductions()
    assert abs(r["Nu"] - 1.0) < 1e-14
    assert abs(r["Re"] - math.sqrt(p.Ra / p.Pr) * abs(c1) / uf) < 1e-10
    # two-valued: left half of the columns at c1, right half at c2
    u = np.full(cav.shape, c1)
    u[:, n // 2:] = c2
    cav.init_fields(T0, [u, np.zeros(cav.shape)])
    r = cav.reductions()
    scale = math.sqrt(p.Ra / p.Pr) / uf
    assert abs(r["Re"] - scale * math.sqrt((c1 ** 2 + c2 ** 2) / 2)) < 1e-10
    assert abs(r["Re_mean"] - scale * (abs(c1) + abs(c2)) / 2) < 1e-10
    assert r["Re"] > r["Re_mean"]          # RMS exceeds the mean for unequal speeds


@pytest.mark.parametrize("name", ["mesh_tanh", "mesh_erf"])
def test_stretched_meshes_shape(name):
    """Both stretched meshes: ends at 0 and 1, exact symmetry, strictly
    increasing, the uniform mesh j/(N+1) in the limit a -> 0, and wall
    clustering whose end-to-centre spacing ratio is the ratio of the stretching
    function's derivatives there: sech^2 for tanh, a Gaussian for erf."""
    mk = getattr(O, name)
    N, a = 401, 1.5
    xi = mk(N, a)
    assert xi[0] == 0.0 and xi[-1] == 1.0
    assert np.all(xi + xi[::-1] == 1.0) and np.all(np.diff(xi) > 0)
    lim = mk(N, 1e-5)
    np.testing.assert_allclose(lim, np.arange(N + 2) / (N + 1), rtol=0, atol=1e-9)
    d = np.diff(xi)
    ratio = d[0] / d[N // 2]
    # derivative of the stretching function at the two intervals' midpoints
    # (midpoint differences are second-order accurate)
    s_end, s_mid = 0.5 / (N + 1) - 0.5, (N // 2 + 0.5) / (N + 1) - 0.5
    if name == "mesh_tanh":
        deriv = lambda s: 1.0 / math.cosh(a * s) ** 2
    else:
        deriv = lambda s: math.exp(-(a * s) ** 2)
    expect = deriv(s_end) / deriv(s_mid)
    assert abs(ratio / expect - 1) < 1e-4, (ratio, expect)

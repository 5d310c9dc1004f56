"""Pins of the oracle's 3-D path (D3Q19 + D3Q7, Sec. 4) to things other than
itself (CPU only).

* Relaxation rates.  With every rate set apart, each family of moments built
  here from monomials of the velocities (orthogonalised by degree) must relax at
  the rate of its physical role: the trace of the second-order tensor at s_e,
  its deviatoric part at s_nu (the viscosity), the third-order heat-flux-like
  and anti-symmetric moments at s_q and s_m, the fourth-order isotropic and
  anisotropic moments at s_eps and s_pi (Sec. 2.1; readings R1, R3).  The
  temperature lattice likewise: first order at q_j, the second-order trace at
  q_e and its anisotropic part at q_nu (R4).
* Shear wave.  w(x, y) = W sin(2 pi x/L) sin(2 pi y/L) between no-slip walls in
  a box tall in z decays as exp(-nu [(2 pi/L_x)^2 + (2 pi/L_y)^2] t), on a
  uniform and a stretched x mesh.
* Steady conduction at Ra -> 0: T linear between the isothermal walls and
  <Nu> = Nu_hot = Nu_cold = 1 (Sec. 4 definitions).
* Volume and wall-plane averages (Eq. (17), Eq. (18), Sec. 4) of manufactured
  fields on a box with different meshes on its three axes, against closed forms.

Each group plants a mistake in the oracle (a wrong entry of the moment-kind
table, a wrong wall weight, exchanged y / z widths) and checks that the pin
catches it.
"""
import math

import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import uniform01

# ---------------------------------------------------------------------------
# relaxation rates of the moment families
# ---------------------------------------------------------------------------

RATES = dict(s_e=0.9, s_eps=1.3, s_q=1.1, s_pi=1.5, s_m=1.7)
Q_RATES = dict(q_e=0.8, q_nu=1.4)


def _gs(v, basis):
    """v with its components along the (already orthogonal) basis removed,
    under the plain inner product over the velocity set."""
    for b in basis:
        v = v - (v @ b) / (b @ b) * b
    return v


def _flow_families(e):
    cx, cy, cz = (e[:, a].astype(float) for a in range(3))
    one = np.ones(len(e))
    c2 = cx * cx + cy * cy + cz * cz
    trace = _gs(c2, [one])
    dev = [cx * cy, cy * cz, cx * cz, cx * cx - cy * cy, cy * cy - cz * cz]
    sym = [_gs(c2 * c, [c]) for c in (cx, cy, cz)]
    anti = [cx * (cy * cy - cz * cz), cy * (cz * cz - cx * cx), cz * (cx * cx - cy * cy)]
    iso = _gs(c2 * c2, [one, trace])
    aniso = [_gs(c2 * (cx * cx - cy * cy), [cx * cx - cy * cy]),
             _gs(c2 * (cy * cy - cz * cz), [cy * cy - cz * cz])]
    return {"s_e": [trace], "s_nu": dev, "s_q": sym, "s_m": anti, "s_eps": [iso],
            "s_pi": aniso}


def _thermal_families(e):
    cx, cy, cz = (e[:, a].astype(float) for a in range(3))
    one = np.ones(len(e))
    c2 = cx * cx + cy * cy + cz * cz
    return {"q_j": [cx, cy, cz], "q_e": [_gs(c2, [one])],
            "q_nu": [cx * cx - cy * cy, cy * cy - cz * cz]}


def _textbook_feq(e, rho, u):
    """Second-order Hermite D3Q19 equilibrium with the textbook weights."""
    sq = (e ** 2).sum(axis=1)
    w = np.array([{0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(s)] for s in sq])
    eu = np.tensordot(e.astype(float), u, axes=1)
    usq = (u * u).sum(axis=0)
    return w[:, None] * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * usq)


def _rate_errors():
    """Largest deviation of (phi(f+) - phi(f_eq)) / (phi(f) - phi(f_eq)) from
    1 - s for every family, on random near-equilibrium states.  The temperature
    populations sum to zero at every node (T = T0), so the buoyancy force
    vanishes; their non-equilibrium parts are random."""
    n = 6
    xi = O.mesh_erf(n, 1.5)
    p = O.Params(Ra=1e6, T_hot=0.0, T_cold=0.0, **RATES, **Q_RATES)
    cav = O.Cavity(xi, xi, xi, params=p)
    size = n ** 3
    e = cav.flow.e
    rho = 1 + 0.05 * (2 * uniform01(size, 71) - 1)
    u = 0.05 * (2 * uniform01(3 * size, 72).reshape(3, size) - 1)
    feq = _textbook_feq(e, rho, u)
    f = feq * (1 + 0.1 * (2 * uniform01(19 * size, 73).reshape(19, size) - 1))
    f = f + (rho - f.sum(0)) / 19          # keep rho: the deviation only
    T = np.zeros(size)
    te = cav.thermal.e.astype(float)
    a_T = cav.par.a_T
    t = np.array([(1 - a_T) / 7] + [(6 + a_T) / 42] * 6)
    uu = np.array([(f * e[:, a, None]).sum(0) / f.sum(0) for a in range(3)])
    geq = t[:, None] * T + 0.5 * np.tensordot(te, uu, axes=1) * T
    g = geq + 0.02 * (2 * uniform01(7 * size, 75).reshape(7, size) - 1)
    g = g + (T - g.sum(0)) / 7
    shape = (19,) + cav.shape
    fp, gp = cav.collide(f.reshape(shape), g.reshape((7,) + cav.shape))
    fp, gp = fp.reshape(19, size), gp.reshape(7, size)
    # the equilibrium of the collided state's own rho, u (both conserved)
    rho_c = f.sum(0)
    u_c = np.array([(f * e[:, a, None]).sum(0) / rho_c for a in range(3)])
    feq_c = _textbook_feq(e, rho_c, u_c)
    geq_c = t[:, None] * T + 0.5 * np.tensordot(te, u_c, axes=1) * T
    rates = dict(RATES, s_nu=cav.par.s_nu, **Q_RATES, q_j=3 - math.sqrt(3))
    worst = {}
    for fams, a, ap, aeq in ((_flow_families(e), f, fp, feq_c),
                             (_thermal_families(cav.thermal.e), g, gp, geq_c)):
        for name, polys in fams.items():
            for phi in polys:
                num = phi @ (ap - aeq)
                den = phi @ (a - aeq)
                err = np.abs(num - (1 - rates[name]) * den).max() / np.abs(den).max()
                worst[name] = max(worst.get(name, 0.0), float(err))
    return worst


def test_every_moment_family_relaxes_at_its_rate():
    worst = _rate_errors()
    assert set(worst) == {"s_e", "s_nu", "s_q", "s_m", "s_eps", "s_pi", "q_j", "q_e", "q_nu"}
    for name, err in worst.items():
        assert err < 1e-12, (name, err)


@pytest.mark.parametrize("index,new", [(9, "pi"), (10, "nu"), (14, "m"), (4, "m"),
                                       (16, "q"), (2, "e"), (1, "eps")])
def test_rate_pin_catches_a_wrong_kind_entry(monkeypatch, index, new):
    kinds = list(O.D3Q19.kinds)
    assert kinds[index] != new
    kinds[index] = new
    monkeypatch.setattr(O.D3Q19, "kinds", kinds)
    worst = _rate_errors()
    assert max(worst.values()) > 1e-3


@pytest.mark.parametrize("index,new", [(4, "nu"), (5, "e"), (1, "e")])
def test_rate_pin_catches_a_wrong_thermal_kind_entry(monkeypatch, index, new):
    kinds = list(O.D3Q7.kinds)
    assert kinds[index] != new
    kinds[index] = new
    monkeypatch.setattr(O.D3Q7, "kinds", kinds)
    worst = _rate_errors()
    assert max(worst.values()) > 1e-3


# ---------------------------------------------------------------------------
# shear wave: the viscosity in 3-D with no-slip walls
# ---------------------------------------------------------------------------


def _shear_wave_rate_error(mesh):
    """w(x, y) = W sin(2 pi x/L_x) sin(2 pi y/L_y) in a 16 x 16 x 128 box (distances
    from the half-way walls): the mid-height amplitude decays at
    nu [(2 pi/L_x)^2 + (2 pi/L_y)^2] until the sound waves from the end walls
    arrive (64 l.u. at c_s: ~110 steps)."""
    N, Nz, nu = 16, 128, 0.1
    xi_x = O.mesh_uniform(N) if mesh == "uniform" else O.mesh_erf(N, 1.0)
    Pr, u_f = 0.71, 0.1 / math.sqrt(3)
    Ra = Pr * (u_f * N / nu) ** 2                # L = N: the uniform y axis
    cav = O.Cavity(xi_x, O.mesh_uniform(N), O.mesh_uniform(Nz),
                   params=O.Params(Ra=Ra, Pr=Pr, T_hot=0.0, T_cold=0.0))
    assert abs(cav.par.nu - nu) < 1e-12
    Xx, Xy = cav.X[0], cav.X[1]
    Lx, Ly = O.characteristic_length(Xx), O.characteristic_length(Xy)
    mx = np.sin(2 * np.pi * (Xx[1:-1] - (Xx[1] - 0.5)) / Lx)
    my = np.sin(2 * np.pi * (Xy[1:-1] - (Xy[1] - 0.5)) / Ly)
    mode = my[:, None] * mx[None, :]
    zero = np.zeros(cav.shape)
    cav.init_fields(zero, u=[zero, zero, np.broadcast_to(1e-3 * mode, cav.shape).copy()])
    wts = cav.W[1][:, None] * cav.W[0][None, :]
    amps, times = [], []
    for _ in range(9):
        cav.step(10)
        w = cav.fields()[1][2][Nz // 2]
        amps.append((wts * w * mode).sum() / (wts * mode * mode).sum())
        times.append(cav.time)
    rate = -np.polyfit(times[1:], np.log(amps[1:]), 1)[0]
    return rate / (nu * ((2 * np.pi / Lx) ** 2 + (2 * np.pi / Ly) ** 2)) - 1


@pytest.mark.parametrize("mesh", ["uniform", "erf"])
def test_3d_shear_wave_decay_gives_the_viscosity(mesh):
    # measured: -0.05% (uniform), +0.13% (stretched x)
    assert abs(_shear_wave_rate_error(mesh)) < (0.01 if mesh == "uniform" else 0.02)


def test_3d_shear_pin_catches_a_wrong_stress_rate(monkeypatch):
    kinds = list(O.D3Q19.kinds)
    kinds[14] = "m"          # p_yz relaxed at the third-order rate
    monkeypatch.setattr(O.D3Q19, "kinds", kinds)
    assert abs(_shear_wave_rate_error("uniform")) > 0.1


# ---------------------------------------------------------------------------
# steady conduction
# ---------------------------------------------------------------------------


def _conduction(mesh, steps=2500):
    N = 8
    xi = O.mesh_uniform(N) if mesh == "uniform" else O.mesh_erf(N, 1.5)
    L = O.characteristic_length(O.lattice_coordinates(xi))
    # alpha = 0.08 keeps a_T = 42 sqrt(3) alpha - 6 inside the D3Q7 range (-6, 1]
    Pr, Ra, alpha = 0.71, 1e-6, 0.08
    Ma = alpha * math.sqrt(Pr * Ra) / L * math.sqrt(3)
    cav = O.Cavity(xi, xi, xi, params=O.Params(Ra=Ra, Pr=Pr, Ma=Ma))
    assert abs(cav.par.alpha - alpha) < 1e-12
    cav.init_fields(np.zeros(cav.shape))
    cav.step(steps)
    return cav


@pytest.mark.parametrize("mesh", ["uniform", "erf"])
def test_3d_steady_conduction_is_linear_with_unit_nusselt(mesh):
    cav = _conduction(mesh)
    rho, u, T = cav.fields()
    X = cav.X[0][1:-1]
    T_lin = 0.5 - (X - (cav.X[0][1] - 0.5)) / cav.L
    np.testing.assert_allclose(T, np.broadcast_to(T_lin, T.shape), atol=1e-8)
    r = cav.reductions()
    for k in ("Nu_hot", "Nu_cold", "Nu"):
        assert abs(r[k] - 1.0) < 1e-8, (k, r[k])


def test_3d_conduction_pin_catches_a_wrong_wall_weight(monkeypatch):
    monkeypatch.setattr(O.D3Q7, "omega", lambda a_T: (6 + a_T) / 20)
    r = _conduction("erf").reductions()
    assert abs(r["Nu_hot"] - 1.0) > 1e-3


# ---------------------------------------------------------------------------
# volume and wall-plane averages on a box with three different meshes
# ---------------------------------------------------------------------------


def _box():
    xi_x, xi_y, xi_z = O.mesh_erf(10, 1.5), O.mesh_uniform(12), O.mesh_tanh(12, 1.2)
    return O.Cavity(xi_x, xi_y, xi_z, params=O.Params(Ra=1e6, Pr=0.71))


def _midpoint_widths(xi):
    """Eq. (18) in lattice units, recomputed from the mesh: X = xi / (xi_1 - xi_0)."""
    X = np.asarray(xi) / (xi[1] - xi[0])
    return 0.5 * (X[2:] - X[:-2]), X


def test_3d_wall_averages_of_manufactured_fields():
    """T = T_hot + (a d + b d^2) h(y, z) near the hot wall, d the distance from
    it: Eq. (17) is exact on quadratics, so Nu_hot = -(L/dT) a <h>, with <h> the
    Eq. (18) average over the wall plane of a product h = 1 + phi(y) psi(z):
    1 + (sum W_y phi)(sum W_z psi) / (sum W_y sum W_z).  Mirror image at the
    cold wall."""
    cav = _box()
    p = cav.p
    Wy, _ = _midpoint_widths(O.mesh_uniform(12))
    Wz, _ = _midpoint_widths(O.mesh_tanh(12, 1.2))
    Xx = cav.X[0]
    phi = 2 * uniform01(12, 81) - 1
    psi = 2 * uniform01(12, 82) - 1
    h = 1 + phi[None, :] * psi[:, None]               # [z, y]
    a, b = -0.004, 0.0007
    d_hot = Xx[1:-1] - (Xx[1] - 0.5)
    d_cold = (Xx[-2] + 0.5) - Xx[1:-1]
    T = np.where(d_hot[None, None, :] < d_cold[None, None, :],
                 p.T_hot + (a * d_hot + b * d_hot ** 2)[None, None, :] * h[:, :, None],
                 p.T_cold - (a * d_cold + b * d_cold ** 2)[None, None, :] * h[:, :, None])
    mean_h = 1 + (Wy @ phi) * (Wz @ psi) / (Wy.sum() * Wz.sum())
    dT = p.T_hot - p.T_cold
    # Eq. (17) measures from the wall (ghost node at -0.5 l.u.): its exact
    # derivative of the quadratic at the wall is a
    expect_hot = -cav.L * a * mean_h / dT
    expect_cold = -cav.L * a * mean_h / dT
    r = _reductions_with_T(cav, T)
    assert abs(r["Nu_hot"] - expect_hot) < 1e-11 * abs(expect_hot)
    assert abs(r["Nu_cold"] - expect_cold) < 1e-11 * abs(expect_cold)


def _reductions_with_T(cav, T):
    cav.init_fields(T - 0.0)
    # equilibrium initialisation keeps T exactly (sum g = T - T_s)
    np.testing.assert_allclose(cav.fields()[2], T, atol=1e-15)
    return cav.reductions()


def test_3d_wall_average_pin_catches_exchanged_widths(monkeypatch):
    cav = _box()
    W1, W2 = cav.W[1].copy(), cav.W[2].copy()
    cav.W[1], cav.W[2] = W2, W1            # y widths on z and z widths on y
    p = cav.p
    phi = 2 * uniform01(12, 81) - 1
    psi = 2 * uniform01(12, 82) - 1
    h = 1 + phi[None, :] * psi[:, None]
    Xx = cav.X[0]
    d_hot = Xx[1:-1] - (Xx[1] - 0.5)
    T = p.T_hot + (-0.004 * d_hot)[None, None, :] * h[:, :, None]
    Wy, _ = _midpoint_widths(O.mesh_uniform(12))
    Wz, _ = _midpoint_widths(O.mesh_tanh(12, 1.2))
    mean_h = 1 + (Wy @ phi) * (Wz @ psi) / (Wy.sum() * Wz.sum())
    expect = -cav.L * -0.004 * mean_h / (p.T_hot - p.T_cold)
    r = _reductions_with_T(cav, T)
    assert abs(r["Nu_hot"] - expect) > 1e-6 * abs(expect)


def test_3d_volume_averages_of_uniform_and_split_flows():
    """Uniform T* and velocity: <Nu> = sqrt(Ra Pr) u* T* + 1, <Re> (RMS, with w)
    and Re_uv (two components) in closed form; velocity split between the
    lower and upper halves of the z range: the volume fractions are the sums of
    the Eq. (18) z widths of each half, recomputed from the mesh."""
    cav = _box()
    p, uf = cav.p, cav.par.u_f
    Tc = np.full(cav.shape, p.T_cold)               # T* = 0: no force, u as given
    c = (0.02 * uf, -0.03 * uf, 0.04 * uf)
    cav.init_fields(Tc, [np.full(cav.shape, v) for v in c])
    r = cav.reductions()
    s = math.sqrt(p.Ra / p.Pr) / uf
    assert abs(r["Nu"] - 1.0) < 1e-14
    assert abs(r["Re"] - s * math.sqrt(sum(v * v for v in c))) < 1e-10
    assert abs(r["Re_uv"] - s * math.hypot(c[0], c[1])) < 1e-10
    Wz, _ = _midpoint_widths(O.mesh_tanh(12, 1.2))
    frac = Wz[:6].sum() / Wz.sum()                  # lower half of the z nodes
    w = np.zeros(cav.shape)
    w[:6] = 0.05 * uf
    w[6:] = -0.01 * uf
    cav.init_fields(Tc, [np.zeros(cav.shape), np.zeros(cav.shape), w])
    r = cav.reductions()
    assert abs(r["Re"] - s * math.sqrt(frac * (0.05 * uf) ** 2 + (1 - frac) * (0.01 * uf) ** 2)) < 1e-10
    assert abs(r["Re_mean"] - s * (frac * 0.05 * uf + (1 - frac) * 0.01 * uf)) < 1e-10
    assert abs(r["Re_uv"]) < 1e-10             # rounding of zero velocities
    # uniform T* > 0 and uniform u (the force shifts only v): <Nu> closed form
    Tstar = 0.3
    Th = np.full(cav.shape, p.T_cold + Tstar * (p.T_hot - p.T_cold))
    cav.init_fields(Th, [np.full(cav.shape, c[0]), np.zeros(cav.shape), np.zeros(cav.shape)])
    r = cav.reductions()
    assert abs(r["Nu"] - (math.sqrt(p.Ra * p.Pr) * (c[0] / uf) * Tstar + 1.0)) < 1e-10
    assert abs(r["mass"] - sum(_midpoint_widths(x)[0].sum() for x in [O.mesh_erf(10, 1.5)]) *
               _midpoint_widths(O.mesh_uniform(12))[0].sum() * Wz.sum()) < 1e-9

"""Plain FP64 CPU oracle of the interpolation-supplemented lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import it; the library never does, and the two
share no code, header, table or constant generator.

Source: Xu, Zhao, Xu & Jiang, "Interpolation-supplemented lattice Boltzmann
simulation of thermal convection on non-uniform meshes", Int. J. Heat Mass
Transfer (2025).  Every function names the passage it follows:

  Sec. 2.1   double-distribution MRT model: D2Q9 / D3Q19 flow populations with
             the printed equilibrium moments and Guo forcing moments, D2Q5 /
             D3Q7 temperature populations with the printed equilibrium moments
             and the a_T <-> alpha relation; collision/streaming split.
  Sec. 2.2   ISLBM: collide locally, stream virtually to x + e_i dt, bring the
             values back to the grid with quadratic (3-point Lagrange)
             interpolation, one axis after the other (virtual nodes).
  Sec. 2.3   half-way bounce-back (no slip), half-way anti-bounce-back
             (isothermal wall), bounce-back (adiabatic wall); uniform mesh
             Eq. (14a,b); error-function mesh; Table 1 length scales; wall
             derivatives Eq. (16)/(17); midpoint-rule average Eq. (18).
  Sec. 3     Ma = 0.1 and the free-fall velocity; steady-state criterion;
             <Nu>, Nu_hot, Nu_middle, <Re>; Richardson extrapolation and GCI.
  Sec. 4     3-D <Nu>, Nu_hot, Nu_cold, <Re>.

Readings taken where the paper is silent, ambiguous or garbled (each is a
parameter below; the defaults are the readings):
  R1  M (D2Q9: Lallemand & Luo rows; D3Q19: d'Humieres et al. rows) and N
      (D2Q5 / D3Q7 standard rows) are not printed.  They are fixed here by
      their polynomial rows; the printed equilibrium and forcing moments pin
      them (tests/test_oracle_pins.py).
  R2  The D2Q9 forcing moment of p_xy is printed as u F_x + v F_y; Guo's
      forcing gives u F_y + v F_x (the D3Q19 vector prints that form).  We use
      u F_y + v F_x.
  R3  Flow rates: s_rho = s_j = 1 (they do not change the result);
      s_e = s_eps (= s_pi in 3-D) = s_nu; s_q (= s_m in 3-D) = 8(2 - s_nu)/(8 - s_nu).
  R4  Thermal rates: q_j = 3 - sqrt(3) is implied by the printed a_T formulas;
      q_e = q_nu = 1.
  R5  Stencil: centred on the target node, {j-1, j, j+1}, moved inwards at the
      ends ({1,2,3} / {N-2,N-1,N}); "upwind" {j-1-c .. j+1-c} is an option.
  R6  Meshes are given in ghost-node form xi_0 .. xi_{N+1}: xi_0 and xi_{N+1}
      sit 1 l.u. beyond the first and last fluid node (the paper's error-function
      mesh already has this form; the uniform mesh of Eq. (14) is written with
      ghost nodes at -1/(2N) and 1 + 1/(2N)).  Walls lie 0.5 l.u. from the
      first and last fluid node; L = X_N - X_1 + 1 (Table 1).
  R7  T0, the reference temperature of the buoyancy force and of T* = (T-T0)/dT,
      is the cold wall, while the temperature populations carry T - T_s with
      T_s the mean wall temperature (walls at +1/2 and -1/2; T* = T + 1/2 lies
      in [0, 1]).  The paper's tables fix both: Table 3's centre values
      T_c = 0.49945 and u_c = -1.2163e-4 are not those of a centro-symmetric
      field (which a mean-wall force reference gives), and Table 2's <Nu> and
      Nu_middle lie 0.26% below Nu_hot, the signature of a convective flux
      u T* evaluated with an offset from the transported temperature (with the
      transported temperature equal to T*, <Nu> = Nu_hot to 1e-4).
  R8  Gravity points along -y: the buoyancy force is +rho g beta (T - T0) y-hat,
      which turns the cell clockwise with the hot wall on the left.
  R9  Nu_middle for even N is evaluated on the face between the two centre
      columns; for odd N on the centre column with a central derivative.
  R10 <Re> uses the root-mean-square speed, sqrt(Ra/Pr) sqrt(<u*^2 + v*^2>_V):
      it reproduces Table 2 (the printed <sqrt(u*^2 + v*^2)>_V, returned as
      Re_mean, is ~27% lower than the tabulated values).  In 3-D |u| includes
      w; the printed two-component form is returned as Re_uv.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ============================================================================
# Lattices (Sec. 2.1)
# ============================================================================


def _opposites(e: np.ndarray) -> np.ndarray:
    """Index of the direction -e_i for every i."""
    return np.array([int(np.where((e == -ei).all(axis=1))[0][0]) for ei in e])


def _matrix(rows, e: np.ndarray) -> np.ndarray:
    """Transformation matrix whose row k is the polynomial rows[k] evaluated on each e_i."""
    return np.array([[float(r(c)) for c in e] for r in rows])


def _sq(c):
    return float(np.dot(c, c))


class FlowLattice:
    """Flow velocity set with its transformation matrix M (reading R1).

    meq(rho, u) returns the printed equilibrium moments m^(eq) (Sec. 2.1);
    mforce(u, F) returns the printed Guo forcing moments M F~ (Sec. 2.1,
    reading R2 for the D2Q9 p_xy entry).  `kinds` names the relaxation rate
    of every moment (reading R3).
    """

    def __init__(self, name, e, rows, kinds, meq, mforce):
        self.name = name
        self.e = np.asarray(e, dtype=np.int64)
        self.q, self.d = self.e.shape
        self.M = _matrix(rows, self.e)
        self.Minv = np.linalg.inv(self.M)
        self.opp = _opposites(self.e)
        self.kinds = kinds
        self.meq = meq
        self.mforce = mforce


class ThermalLattice:
    """Temperature velocity set with its transformation matrix N (reading R1).

    neq(T, u, a_T) returns the printed n^(eq) (Sec. 2.1).  a_T_of_alpha is the
    printed diffusivity relation; omega(a_T) the printed anti-bounce-back
    weight (Sec. 2.3).
    """

    def __init__(self, name, e, rows, kinds, neq, a_T_of_alpha, omega):
        self.name = name
        self.e = np.asarray(e, dtype=np.int64)
        self.q, self.d = self.e.shape
        self.N = _matrix(rows, self.e)
        self.Ninv = np.linalg.inv(self.N)
        self.opp = _opposites(self.e)
        self.kinds = kinds
        self.neq = neq
        self.a_T_of_alpha = a_T_of_alpha
        self.omega = omega


# ---- D2Q9 (Lallemand & Luo moment basis: rho, e, eps, jx, qx, jy, qy, pxx, pxy)
_E_D2Q9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_ROWS_D2Q9 = [
    lambda c: 1,
    lambda c: -4 + 3 * _sq(c),
    lambda c: 4 - 10.5 * _sq(c) + 4.5 * _sq(c) ** 2,
    lambda c: c[0],
    lambda c: (-5 + 3 * _sq(c)) * c[0],
    lambda c: c[1],
    lambda c: (-5 + 3 * _sq(c)) * c[1],
    lambda c: c[0] ** 2 - c[1] ** 2,
    lambda c: c[0] * c[1],
]


def _meq_d2q9(rho, u):
    """Printed D2Q9 equilibrium moments, Sec. 2.1."""
    ux, uy = u
    usq = ux * ux + uy * uy
    return [rho, rho * (-2 + 3 * usq), rho * (1 - 3 * usq), rho * ux, -rho * ux,
            rho * uy, -rho * uy, rho * (ux * ux - uy * uy), rho * ux * uy]


def _mforce_d2q9(u, F):
    """Printed D2Q9 Guo forcing moments M F~, Sec. 2.1 (p_xy entry: reading R2)."""
    ux, uy = u
    Fx, Fy = F
    uF = ux * Fx + uy * Fy
    zero = 0 * uF
    return [zero, 6 * uF, -6 * uF, Fx + zero, -Fx + zero, Fy + zero, -Fy + zero,
            2 * ux * Fx - 2 * uy * Fy, ux * Fy + uy * Fx]


D2Q9 = FlowLattice("D2Q9", _E_D2Q9, _ROWS_D2Q9,
                   ["rho", "e", "eps", "j", "q", "j", "q", "nu", "nu"],
                   _meq_d2q9, _mforce_d2q9)

# ---- D3Q19 (d'Humieres et al. moment basis)
_E_D3Q19 = [(0, 0, 0),
            (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
            (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
            (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
            (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
_ROWS_D3Q19 = [
    lambda c: 1,
    lambda c: -30 + 19 * _sq(c),
    lambda c: 12 - 26.5 * _sq(c) + 10.5 * _sq(c) ** 2,
    lambda c: c[0],
    lambda c: (-9 + 5 * _sq(c)) * c[0],
    lambda c: c[1],
    lambda c: (-9 + 5 * _sq(c)) * c[1],
    lambda c: c[2],
    lambda c: (-9 + 5 * _sq(c)) * c[2],
    lambda c: 3 * c[0] ** 2 - _sq(c),
    lambda c: (-5 + 3 * _sq(c)) * (3 * c[0] ** 2 - _sq(c)),
    lambda c: c[1] ** 2 - c[2] ** 2,
    lambda c: (-5 + 3 * _sq(c)) * (c[1] ** 2 - c[2] ** 2),
    lambda c: c[0] * c[1],
    lambda c: c[1] * c[2],
    lambda c: c[0] * c[2],
    lambda c: (c[1] ** 2 - c[2] ** 2) * c[0],
    lambda c: (c[2] ** 2 - c[0] ** 2) * c[1],
    lambda c: (c[0] ** 2 - c[1] ** 2) * c[2],
]


def _meq_d3q19(rho, u):
    """Printed D3Q19 equilibrium moments, Sec. 2.1."""
    ux, uy, uz = u
    usq = ux * ux + uy * uy + uz * uz
    p1 = 2 * ux * ux - uy * uy - uz * uz
    p2 = uy * uy - uz * uz
    zero = 0 * rho
    return [rho, rho * (-11 + 19 * usq), rho * (3 - 5.5 * usq),
            rho * ux, -2.0 / 3.0 * rho * ux, rho * uy, -2.0 / 3.0 * rho * uy,
            rho * uz, -2.0 / 3.0 * rho * uz,
            rho * p1, -0.5 * rho * p1, rho * p2, -0.5 * rho * p2,
            rho * ux * uy, rho * uy * uz, rho * ux * uz, zero, zero, zero]


def _mforce_d3q19(u, F):
    """Printed D3Q19 Guo forcing moments M F~, Sec. 2.1."""
    ux, uy, uz = u
    Fx, Fy, Fz = F
    uF = ux * Fx + uy * Fy + uz * Fz
    zero = 0 * uF
    return [zero, 38 * uF, -11 * uF,
            Fx + zero, -2.0 / 3.0 * Fx + zero, Fy + zero, -2.0 / 3.0 * Fy + zero,
            Fz + zero, -2.0 / 3.0 * Fz + zero,
            4 * ux * Fx - 2 * uy * Fy - 2 * uz * Fz, -2 * ux * Fx + uy * Fy + uz * Fz,
            2 * uy * Fy - 2 * uz * Fz, -uy * Fy + uz * Fz,
            ux * Fy + uy * Fx, uy * Fz + uz * Fy, ux * Fz + uz * Fx, zero, zero, zero]


D3Q19 = FlowLattice("D3Q19", _E_D3Q19, _ROWS_D3Q19,
                    ["rho", "e", "eps", "j", "q", "j", "q", "j", "q",
                     "nu", "pi", "nu", "pi", "nu", "nu", "nu", "m", "m", "m"],
                    _meq_d3q19, _mforce_d3q19)

# ---- D2Q5 / D3Q7 temperature lattices
_E_D2Q5 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)]
_ROWS_D2Q5 = [lambda c: 1, lambda c: c[0], lambda c: c[1],
              lambda c: -4 + 5 * _sq(c), lambda c: c[0] ** 2 - c[1] ** 2]


def _neq_d2q5(T, u, a_T):
    """Printed D2Q5 equilibrium moments [T, uT, vT, a_T T, 0], Sec. 2.1."""
    return [T, u[0] * T, u[1] * T, a_T * T, 0 * T]


D2Q5 = ThermalLattice("D2Q5", _E_D2Q5, _ROWS_D2Q5, ["T", "j", "j", "e", "nu"], _neq_d2q5,
                      a_T_of_alpha=lambda alpha: 20 * math.sqrt(3) * alpha - 4,
                      omega=lambda a_T: (4 + a_T) / 10)

_E_D3Q7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
_ROWS_D3Q7 = [lambda c: 1, lambda c: c[0], lambda c: c[1], lambda c: c[2],
              lambda c: -6 + 7 * _sq(c), lambda c: 3 * c[0] ** 2 - _sq(c),
              lambda c: c[1] ** 2 - c[2] ** 2]


def _neq_d3q7(T, u, a_T):
    """Printed D3Q7 equilibrium moments [T, uT, vT, wT, a_T T, 0, 0], Sec. 2.1."""
    return [T, u[0] * T, u[1] * T, u[2] * T, a_T * T, 0 * T, 0 * T]


D3Q7 = ThermalLattice("D3Q7", _E_D3Q7, _ROWS_D3Q7, ["T", "j", "j", "j", "e", "nu", "nu"],
                      _neq_d3q7,
                      a_T_of_alpha=lambda alpha: 42 * math.sqrt(3) * alpha - 6,
                      omega=lambda a_T: (6 + a_T) / 21)

# ============================================================================
# Meshes and length scales (Sec. 2.3, Table 1)
# ============================================================================


def mesh_uniform(N: int) -> np.ndarray:
    """Eq. (14b) nodes (j - 0.5)/N with ghost nodes 1/N beyond the ends (reading R6)."""
    j = np.arange(N + 2, dtype=np.float64)
    return (j - 0.5) / N


def _mirror(xi: np.ndarray) -> np.ndarray:
    """Make xi exactly symmetric, xi_{N+1-j} = 1 - xi_j."""
    n = len(xi)
    out = xi.copy()
    for j in range(n // 2, n):
        out[j] = 1.0 - xi[n - 1 - j]
    return out


def mesh_erf(N: int, a: float = 1.5) -> np.ndarray:
    """Error-function stretched mesh, Sec. 2.3: y_j = (erf[a(j/(N+1) - 1/2)]/erf(a/2) + 1)/2."""
    xi = np.array([0.5 * (math.erf(a * (j / (N + 1) - 0.5)) / math.erf(a / 2) + 1.0)
                   for j in range(N + 2)])
    return _mirror(xi)


def mesh_tanh(N: int, a: float = 1.5) -> np.ndarray:
    """Hyperbolic-tangent analogue of the error-function mesh (same form, tanh for erf)."""
    xi = np.array([0.5 * (math.tanh(a * (j / (N + 1) - 0.5)) / math.tanh(a / 2) + 1.0)
                   for j in range(N + 2)])
    return _mirror(xi)


def lattice_coordinates(xi: np.ndarray) -> np.ndarray:
    """X_j in lattice units: 1 l.u. = xi_1 - xi_0, the minimal resolution of Table 1.

    A mesh whose coordinates are integers to rounding is the uniform mesh of
    Eq. (14); its lattice coordinates are made exact integers.
    """
    X = (xi - xi[0]) / (xi[1] - xi[0])
    if np.abs(X - np.round(X)).max() < 1e-9:
        X = np.round(X)
    return X


def cell_widths(X: np.ndarray) -> np.ndarray:
    """Midpoint-rule weights of Eq. (18): W_j = (X_{j+1} - X_{j-1})/2, j = 1..N."""
    return 0.5 * (X[2:] - X[:-2])


def characteristic_length(X: np.ndarray) -> float:
    """Effective cavity height in l.u. (Table 1): distance between the two half-way walls."""
    return float(X[-2] - X[1] + 1.0)


def mesh_quality(xi: np.ndarray):
    """Maximum growth rate of adjacent spacings and maximum cell aspect ratio (Sec. 2.3)
    of the square tensor-product mesh built from xi on both axes."""
    d = np.diff(xi)
    growth = np.maximum(d[1:] / d[:-1], d[:-1] / d[1:]).max()
    aspect = d.max() / d.min()
    return float(growth), float(aspect)


# ============================================================================
# Quadratic interpolation tables (Sec. 2.2)
# ============================================================================


@dataclass
class AxisTable:
    """Per-axis, per-direction (c = +1 / -1) stencil data for the fluid nodes j = 1..N.

    base[j-1] is the 0-based fluid index of the first of the three stencil
    nodes, w[j-1] the Lagrange weights, wall[j-1] is True where the departure
    point X_j - c lies beyond a half-way wall (bounce-back instead).
    """
    base: np.ndarray
    w: np.ndarray
    wall: np.ndarray


def lagrange_weights(nodes, x):
    """Quadratic Lagrange basis l_m(x) = prod_{n != m} (x - x_n)/(x_m - x_n) on three nodes."""
    out = []
    for m in range(3):
        v = 1.0
        for n in range(3):
            if n != m:
                v *= (x - nodes[n]) / (nodes[m] - nodes[n])
        out.append(v)
    return out


def interpolation_table(X: np.ndarray, c: int, stencil: str = "centred") -> AxisTable:
    """Stencils and weights that bring the virtually streamed values back to node j.

    The post-collision value of node k moves to X_k + c (Sec. 2.2); the value at
    X_j is the quadratic interpolant through three such points, which equals
    the Lagrange interpolant of the node values evaluated at the departure
    point X_j - c.  Reading R5 fixes the stencil.
    """
    N = len(X) - 2
    base = np.zeros(N, dtype=np.int64)
    w = np.zeros((N, 3))
    wall = np.zeros(N, dtype=bool)
    for j in range(1, N + 1):
        if (j == 1 and c == +1) or (j == N and c == -1):
            wall[j - 1] = True
            continue
        b = j - 1 if stencil == "centred" else j - 1 - c
        b = min(max(b, 1), N - 2)
        base[j - 1] = b - 1
        w[j - 1] = lagrange_weights(X[b:b + 3], X[j] - c)
    return AxisTable(base, w, wall)


def interpolate_axis(values: np.ndarray, axis: int, tab: AxisTable) -> np.ndarray:
    """out[.., j, ..] = sum_k w[j,k] values[.., base[j]+k, ..] along `axis` (wall entries: 0)."""
    idx = tab.base[:, None] + np.arange(3)[None, :]            # (N, 3)
    gathered = np.take(values, idx, axis=axis)                  # axis -> (N, 3)
    shape = [1] * gathered.ndim
    shape[axis] = tab.w.shape[0]
    shape[axis + 1] = 3
    return (gathered * tab.w.reshape(shape)).sum(axis=axis + 1)


# ============================================================================
# Parameters (Sec. 2.1, Sec. 3)
# ============================================================================


@dataclass
class Params:
    """Physical and numerical parameters.  None means "use the reading's default"."""
    Ra: float
    Pr: float = 0.71
    Ma: float = 0.1
    T_hot: float = 0.5
    T_cold: float = -0.5
    T0: float | None = None          # None: the cold wall (reading R7)
    s_rho: float = 1.0
    s_j: float = 1.0
    s_e: float | None = None
    s_eps: float | None = None
    s_q: float | None = None
    s_pi: float | None = None
    s_m: float | None = None
    q_T: float = 1.0
    q_j: float | None = None
    q_e: float = 1.0
    q_nu: float = 1.0
    stencil: str = "centred"


@dataclass
class Derived:
    L: float
    u_f: float
    nu: float
    alpha: float
    gbeta: float
    s_nu: float
    a_T: float
    omega: float
    S: np.ndarray = field(repr=False)
    Q: np.ndarray = field(repr=False)


def derive(p: Params, L: float, flow: FlowLattice, thermal: ThermalLattice) -> Derived:
    """Lattice-unit parameters.

    u_f = Ma c_s with c_s = 1/sqrt(3) (Sec. 3); from the scalings and
    Ra = g beta dT H^3/(nu alpha), Pr = nu/alpha (Sec. 2.1) with H = L l.u. and
    dT = 1: nu = u_f L sqrt(Pr/Ra), alpha = u_f L / sqrt(Pr Ra), g beta = u_f^2 / L.
    """
    u_f = p.Ma / math.sqrt(3.0)
    nu = u_f * L * math.sqrt(p.Pr / p.Ra)
    alpha = u_f * L / math.sqrt(p.Pr * p.Ra)
    gbeta = u_f * u_f / L
    s_nu = 1.0 / (3.0 * nu + 0.5)
    magic = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)          # reading R3
    rate = {"rho": p.s_rho, "j": p.s_j,
            "e": s_nu if p.s_e is None else p.s_e,
            "eps": s_nu if p.s_eps is None else p.s_eps,
            "q": magic if p.s_q is None else p.s_q,
            "nu": s_nu,
            "pi": s_nu if p.s_pi is None else p.s_pi,
            "m": magic if p.s_m is None else p.s_m}
    S = np.array([rate[k] for k in flow.kinds])
    a_T = thermal.a_T_of_alpha(alpha)
    q_j = (3.0 - math.sqrt(3.0)) if p.q_j is None else p.q_j   # reading R4
    qrate = {"T": p.q_T, "j": q_j, "e": p.q_e, "nu": p.q_nu}
    Q = np.array([qrate[k] for k in thermal.kinds])
    return Derived(L, u_f, nu, alpha, gbeta, s_nu, a_T, thermal.omega(a_T), S, Q)


# ============================================================================
# The cavity solver (Sec. 2.1 - 2.3, Sec. 3, Sec. 4)
# ============================================================================


class Cavity:
    """Side-heated cavity: hot wall at x = 0, cold wall at x = 1, all other walls
    adiabatic, no slip everywhere (Sec. 3, Sec. 4).

    Arrays are indexed [population, (z,) y, x]; axis a of the lattice (x = 0,
    y = 1, z = 2) is array axis -(a+1).
    """

    def __init__(self, xi_x, xi_y, xi_z=None, params: Params | None = None):
        self.p = params if params is not None else Params(Ra=1e6)
        self.T0 = self.p.T_cold if self.p.T0 is None else self.p.T0
        self.Ts = 0.5 * (self.p.T_hot + self.p.T_cold)
        meshes = [np.asarray(xi_x, float), np.asarray(xi_y, float)]
        if xi_z is not None:
            meshes.append(np.asarray(xi_z, float))
        self.d = len(meshes)
        self.flow = D2Q9 if self.d == 2 else D3Q19
        self.thermal = D2Q5 if self.d == 2 else D3Q7
        self.X = [lattice_coordinates(m) for m in meshes]
        self.n = [len(X) - 2 for X in self.X]                 # fluid nodes per axis
        self.shape = tuple(reversed(self.n))                   # (z,) y, x
        self.W = [cell_widths(X) for X in self.X]
        self.L = characteristic_length(self.X[1])              # cavity height H
        self.par = derive(self.p, self.L, self.flow, self.thermal)
        self.tables = [{c: interpolation_table(X, c, self.p.stencil) for c in (+1, -1)}
                       for X in self.X]
        self.f = None
        self.g = None
        self.time = 0

    # ---- helpers ----------------------------------------------------------
    def _axis(self, a: int) -> int:
        return self.d - a   # +1 for the population index: x -> last array axis

    def _bcast(self, vec: np.ndarray, a: int) -> np.ndarray:
        """Reshape a per-axis vector to broadcast along lattice axis a of a field."""
        shape = [1] * self.d
        shape[self.d - 1 - a] = len(vec)
        return vec.reshape(shape)

    # ---- equilibria and macroscopic quantities (Sec. 2.1) -----------------
    def equilibrium(self, rho, u, theta):
        """f^eq = M^-1 m^eq(rho, u) and g^eq = N^-1 n^eq(theta, u), theta = T - T_s (R7)."""
        meq = np.array(self.flow.meq(rho, u))
        neq = np.array(self.thermal.neq(theta, u, self.par.a_T))
        f = np.tensordot(self.flow.Minv, meq, axes=1)
        g = np.tensordot(self.thermal.Ninv, neq, axes=1)
        return f, g

    def init_fields(self, T, u=None, rho=None):
        """Equilibrium initialisation from given T (internal convention) and u."""
        T = np.asarray(T, float).reshape(self.shape)
        if u is None:
            u = [np.zeros(self.shape) for _ in range(self.d)]
        if rho is None:
            rho = np.ones(self.shape)
        self.f, self.g = self.equilibrium(rho, [np.asarray(c, float).reshape(self.shape) for c in u],
                                          T - self.Ts)
        self.time = 0

    def init_populations(self, f, g):
        """Pre-collision populations; the temperature populations carry T - T_s (R7)."""
        self.f = np.array(f, dtype=np.float64).reshape((self.flow.q,) + self.shape)
        self.g = np.array(g, dtype=np.float64).reshape((self.thermal.q,) + self.shape)
        self.time = 0

    def macroscopic(self, f, g):
        """rho = sum f, theta = T - T_s = sum g, F = rho g beta (T - T0) y-hat (R7, R8),
        u = (sum e f + F/2)/rho (Sec. 2.1).  Returns rho, u, theta, F."""
        rho = f.sum(axis=0)
        theta = g.sum(axis=0)
        F = [np.zeros(self.shape) for _ in range(self.d)]
        F[1] = rho * self.par.gbeta * (theta + self.Ts - self.T0)
        u = [(np.tensordot(self.flow.e[:, a].astype(float), f, axes=1) + 0.5 * F[a]) / rho
             for a in range(self.d)]
        return rho, u, theta, F

    # ---- collision (Sec. 2.1, collision steps) ----------------------------
    def collide(self, f, g):
        """f+ = f - M^-1 S (m - m^eq) + F',  F' = M^-1 (I - S/2) M F~;
        g+ = g - N^-1 Q (n - n^eq)."""
        rho, u, theta, F = self.macroscopic(f, g)
        M, Minv, S = self.flow.M, self.flow.Minv, self.par.S
        m = np.tensordot(M, f, axes=1)
        meq = np.array(self.flow.meq(rho, u))
        MF = np.array(self.flow.mforce(u, F))
        relax = S.reshape((-1,) + (1,) * self.d)
        fpost = f - np.tensordot(Minv, relax * (m - meq), axes=1) \
            + np.tensordot(Minv, (1.0 - relax / 2.0) * MF, axes=1)
        Nm, Ninv, Q = self.thermal.N, self.thermal.Ninv, self.par.Q
        n = np.tensordot(Nm, g, axes=1)
        neq = np.array(self.thermal.neq(theta, u, self.par.a_T))
        qrel = Q.reshape((-1,) + (1,) * self.d)
        gpost = g - np.tensordot(Ninv, qrel * (n - neq), axes=1)
        return fpost, gpost

    # ---- virtual streaming, interpolation, walls (Sec. 2.2, 2.3) ----------
    def _stream_one(self, val: np.ndarray, e_i) -> np.ndarray:
        """Interpolate one post-collision population back to the nodes, axis by axis."""
        for a in range(self.d):
            c = int(e_i[a])
            if c != 0:
                val = interpolate_axis(val, self._axis(a) - 1, self.tables[a][c])
        return val

    def _wall_mask(self, e_i):
        """Nodes whose departure point crosses a wall along any moving axis,
        and the axis (x first) that decides the thermal condition."""
        mask = np.zeros(self.shape, dtype=bool)
        for a in range(self.d):
            c = int(e_i[a])
            if c != 0:
                mask = mask | self._bcast(self.tables[a][c].wall, a)
        return mask

    def stream(self, fpost, gpost):
        """f_i(x, t+dt) from the interpolated virtual streaming, or half-way
        bounce-back f_i = f_ibar+ where the departure point lies behind a wall.
        g: anti-bounce-back g_i = -g_ibar+ + omega (T_w - T_s) on the isothermal x-walls,
        bounce-back g_i = g_ibar+ on the adiabatic walls (Sec. 2.3)."""
        fl, th = self.flow, self.thermal
        fnew = np.empty_like(fpost)
        for i in range(fl.q):
            val = self._stream_one(fpost[i], fl.e[i])
            mask = self._wall_mask(fl.e[i])
            fnew[i] = np.where(mask, fpost[fl.opp[i]], val)
        gnew = np.empty_like(gpost)
        for i in range(th.q):
            e_i = th.e[i]
            val = self._stream_one(gpost[i], e_i)
            mask = self._wall_mask(e_i)
            if e_i[0] != 0:       # x-directed: isothermal walls
                T_w = self.p.T_hot if e_i[0] == +1 else self.p.T_cold
                wallval = -gpost[th.opp[i]] + self.par.omega * (T_w - self.Ts)
            else:                 # y- or z-directed: adiabatic walls
                wallval = gpost[th.opp[i]]
            gnew[i] = np.where(mask, wallval, val)
        return fnew, gnew

    def step(self, n: int = 1):
        """n ISLBM cycles: collide -> virtual stream -> interpolate -> walls (Sec. 2.2)."""
        for _ in range(n):
            fpost, gpost = self.collide(self.f, self.g)
            self.f, self.g = self.stream(fpost, gpost)
            self.time += 1

    # ---- diagnostics (Sec. 2.3, Sec. 3, Sec. 4) ---------------------------
    def fields(self):
        """rho, u (list per axis), T at the current time (in the units of T_hot, T_cold)."""
        rho, u, theta, _ = self.macroscopic(self.f, self.g)
        return rho, u, theta + self.Ts

    def post_collision(self):
        return self.collide(self.f, self.g)

    def volume_weights(self) -> np.ndarray:
        w = np.ones(self.shape)
        for a in range(self.d):
            w = w * self._bcast(self.W[a], a)
        return w

    def wall_derivative(self, T: np.ndarray, side: str) -> np.ndarray:
        """dT/dX (per l.u.) at the x = 0 ('hot') or x = 1 ('cold') wall by Eq. (17)
        with Delta = 1 l.u. and q = (X_2 - X_1)/(X_1 - X_0) (Eq. (16) when q = 1)."""
        X = self.X[0]
        if side == "hot":
            q = (X[2] - X[1]) / (X[1] - X[0])
            Tw, T1, T2 = self.p.T_hot, T[..., 0], T[..., 1]
            return (-4 * q * (q + 1) * Tw + (2 * q + 1) ** 2 * T1 - T2) / (q * (2 * q + 1))
        q = (X[-2] - X[-3]) / (X[-1] - X[-2])
        Tw, T1, T2 = self.p.T_cold, T[..., -1], T[..., -2]
        return (4 * q * (q + 1) * Tw - (2 * q + 1) ** 2 * T1 + T2) / (q * (2 * q + 1))

    def reductions(self):
        """<Nu>, Nu_hot, Nu_cold, Nu_middle (2-D), <Re> (R10), mass, kinetic energy (Sec. 3, Sec. 4).

        <phi>_V = sum phi prod W / sum prod W (Eq. (18) on every axis, divided by
        the cavity volume, L^d for the square cavity); u* = u/u_f,
        T* = (T - T0)/dT with dT = T_hot - T_cold; x* = X/L.
        """
        rho, u, T = self.fields()
        par, p, L, d = self.par, self.p, self.L, self.d
        dT = p.T_hot - p.T_cold
        Ts = (T - self.T0) / dT
        us = [c / par.u_f for c in u]
        Wv = self.volume_weights()
        vol = float(Wv.sum())           # L^d for the square / cubic cavity
        out = {}
        out["Nu"] = math.sqrt(p.Ra * p.Pr) * float((Wv * us[0] * Ts).sum()) / vol + 1.0
        speed2 = sum(c * c for c in us)
        out["Re"] = math.sqrt(p.Ra / p.Pr) * math.sqrt(float((Wv * speed2).sum()) / vol)
        out["Re_mean"] = math.sqrt(p.Ra / p.Pr) * float((Wv * np.sqrt(speed2)).sum()) / vol
        out["Re_uv"] = math.sqrt(p.Ra / p.Pr) * math.sqrt(
            float((Wv * (us[0] ** 2 + us[1] ** 2)).sum()) / vol)
        out["mass"] = float((Wv * rho).sum())
        out["ke"] = float((Wv * sum(c * c for c in u)).sum()) * 0.5
        # wall-plane weights: every axis but x
        Wp = np.ones(self.shape[:-1])
        for a in range(1, d):
            shape = [1] * (d - 1)
            shape[d - 1 - a] = len(self.W[a])
            Wp = Wp * self.W[a].reshape(shape)
        area = float(Wp.sum())          # L^(d-1) for the square / cubic cavity
        # Nu = -<dT*/dx*>, dT*/dx* = (L/dT) dT/dX
        for side in ("hot", "cold"):
            dTdX = self.wall_derivative(T, side)
            out["Nu_" + side] = -float((Wp * dTdX).sum()) * L / dT / area
        if d == 2:
            out["Nu_middle"] = self._nu_middle(us, Ts, Wp)
        return out

    def _nu_middle(self, us, Ts, Wy) -> float:
        """<sqrt(Ra Pr) u* T* - dT*/dx*> on the vertical centre line x* = 1/2 (reading R9)."""
        X, L, p = self.X[0], self.L, self.p
        N = self.n[0]
        conv = math.sqrt(p.Ra * p.Pr) * us[0] * Ts
        if N % 2 == 0:
            m = N // 2 - 1                    # 0-based left centre column
            flux = 0.5 * (conv[:, m] + conv[:, m + 1]) \
                - L * (Ts[:, m + 1] - Ts[:, m]) / (X[m + 2] - X[m + 1])
        else:
            m = (N + 1) // 2 - 1
            flux = conv[:, m] - L * (Ts[:, m + 1] - Ts[:, m - 1]) / (X[m + 2] - X[m])
        return float((Wy * flux).sum()) / L


# ============================================================================
# Steady state, convergence studies (Sec. 3)
# ============================================================================


def steady_change(u_new, u_old, T_new, T_old):
    """Relative changes of the steady-state criterion (Sec. 3): sum |u(t+2000) - u(t)|_2
    over sum |u(t)|_2, and sum |T(t+2000) - T(t)| over sum |T(t)|."""
    du = np.sqrt(sum((a - b) ** 2 for a, b in zip(u_new, u_old))).sum()
    un = np.sqrt(sum(b ** 2 for b in u_old)).sum()
    dT = np.abs(T_new - T_old).sum()
    Tn = np.abs(T_old).sum()
    return float(du / un), float(dT / Tn)


def richardson(F_coarse, F_medium, F_fine, r=2.0):
    """Observed order p and extrapolated value F(1/inf) (Sec. 3, Richardson extrapolation)."""
    p = math.log(abs((F_coarse - F_medium) / (F_medium - F_fine))) / math.log(r)
    rp = r ** p
    return p, (rp * F_fine - F_medium) / (rp - 1.0)


def gci_fine(F_medium, F_fine, p, r=2.0, Fs=1.25):
    """Grid Convergence Index of the fine mesh in percent (Sec. 3)."""
    return Fs / (r ** p - 1.0) * abs((F_fine - F_medium) / F_fine) * 100.0

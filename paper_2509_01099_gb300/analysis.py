"""Grid-convergence analysis of solver results (Sec. 3).

Three meshes refined by a constant ratio r give the observed order of a
quantity, its Richardson-extrapolated value on an infinitely fine mesh and
the Grid Convergence Index (safety factor 1.25) of the finest mesh.  Host
arithmetic on a handful of numbers; no device work.
"""
from __future__ import annotations

import math


def observed_order(coarse: float, medium: float, fine: float, ratio: float = 2.0) -> float:
    """p from the ratio of successive differences: (f_c - f_m)/(f_m - f_f) = r^p."""
    return math.log(abs((coarse - medium) / (medium - fine))) / math.log(ratio)


def extrapolate(medium: float, fine: float, order: float, ratio: float = 2.0) -> float:
    """Value on an infinitely fine mesh: the fine value plus its remaining error."""
    return fine + (fine - medium) / (ratio ** order - 1.0)


def gci_percent(medium: float, fine: float, order: float, ratio: float = 2.0,
                safety: float = 1.25) -> float:
    """Grid Convergence Index of the fine mesh, in percent."""
    return 100.0 * safety * abs((fine - medium) / fine) / (ratio ** order - 1.0)


def convergence_table(values, ratio: float = 2.0) -> dict:
    """{name: (coarse, medium, fine)} -> {name: {values, p, inf, gci_percent}}."""
    out = {}
    for name, (c, m, f) in values.items():
        try:
            p = observed_order(c, m, f, ratio)
            out[name] = {"values": [c, m, f], "p": p, "inf": extrapolate(m, f, p, ratio),
                         "gci_percent": gci_percent(m, f, p, ratio)}
        except (ValueError, ZeroDivisionError):
            out[name] = {"values": [c, m, f], "p": None, "inf": None, "gci_percent": None}
    return out


# ---------------------------------------------------------------------------
# Post-processing diagnostics of steady 2-D fields (Sec. 3): mid-height band
# profiles, boundary-layer thicknesses by the 99% and slope methods, their
# Rayleigh-number scaling, and the velocity divergence.  Coordinates are the
# nondimensional node positions x* in (0, 1); fields are [ny][nx] arrays.
# ---------------------------------------------------------------------------

import numpy as np  # noqa: E402


def node_positions(xi) -> np.ndarray:
    """x* of the fluid nodes of a ghost-node mesh (walls half a lattice unit outside)."""
    xi = np.asarray(xi, dtype=np.float64)
    X = (xi - xi[0]) / (xi[1] - xi[0])            # lattice units, ghost at 0
    L = X[-2] - X[1] + 1.0
    return (X[1:-1] - X[1] + 0.5) / L


def band_profiles(field, y_star, band=(0.4, 0.6), weights=None):
    """Average of a [ny][nx] field over the rows with band[0] <= y* <= band[1]."""
    rows = (y_star >= band[0]) & (y_star <= band[1])
    w = np.ones(rows.sum()) if weights is None else np.asarray(weights)[rows]
    return (np.asarray(field)[rows] * w[:, None]).sum(axis=0) / w.sum()


def _first_crossing(x, f, level):
    """x where f first reaches `level` moving away from x[0] (linear interpolation)."""
    for k in range(1, len(f)):
        if (f[k - 1] - level) * (f[k] - level) <= 0 and f[k] != f[k - 1]:
            return x[k - 1] + (level - f[k - 1]) * (x[k] - x[k - 1]) / (f[k] - f[k - 1])
    return float("nan")


def boundary_layers(x, T, v, T_wall=1.0):
    """Thermal and velocity boundary-layer thicknesses at the hot wall x* = 0 from
    band-averaged profiles T*(x*), v*(x*):
      99% method: delta_T where T* has covered 99% of the wall-to-core difference
      (core: the value at x* = 1/2); delta_V where v* first reaches 99% of its maximum.
      slope method: delta_T = (T_wall - T_core) / |dT*/dx*| at the wall;
      delta_V = v_max / |dv*/dx*| at the wall (no slip: v = 0 at x* = 0)."""
    x, T, v = (np.asarray(a, dtype=np.float64) for a in (x, T, v))
    half = np.argmin(np.abs(x - 0.5))
    T_core = T[half]
    near = x < 0.5
    xs, Ts, vs = np.concatenate(([0.0], x[near])), np.concatenate(([T_wall], T[near])), \
        np.concatenate(([0.0], v[near]))
    dT99 = _first_crossing(xs, Ts, T_wall - 0.99 * (T_wall - T_core))
    imax = int(np.argmax(vs))
    dV99 = _first_crossing(xs[:imax + 1], vs[:imax + 1], 0.99 * vs[imax])
    # one-sided wall gradients from the wall value and the first two nodes (quadratic)
    h1, h2 = xs[1], xs[2]
    def wall_slope(f0, f1, f2):
        return (f1 - f0) * h2 / (h1 * (h2 - h1)) - (f2 - f0) * h1 / (h2 * (h2 - h1))
    gT = wall_slope(Ts[0], Ts[1], Ts[2])
    gV = wall_slope(vs[0], vs[1], vs[2])
    return {"delta_T_99": dT99, "delta_V_99": dV99,
            "delta_T_slope": abs(T_wall - T_core) / abs(gT), "delta_V_slope": vs[imax] / abs(gV),
            "T_core": T_core, "v_max": vs[imax]}


def power_law(ra, delta):
    """Exponent p and prefactor c of delta = c Ra^p (least squares in log-log)."""
    p, lc = np.polyfit(np.log(np.asarray(ra, float)), np.log(np.asarray(delta, float)), 1)
    return float(p), float(np.exp(lc))


def divergence_2d(u, v, x, y):
    """du/dx + dv/dy on the non-uniform node positions (second-order centred
    differences in the interior, one-sided at the first and last nodes)."""
    return np.gradient(np.asarray(u, float), np.asarray(x, float), axis=1) + \
        np.gradient(np.asarray(v, float), np.asarray(y, float), axis=0)


# ---------------------------------------------------------------------------
# Centre values, 3-D profiles and divergence statistics (Sec. 3, Sec. 4)
# ---------------------------------------------------------------------------


def _centre_pair(x):
    """Indices (i0, i1) of the node(s) at x* = 1/2 (i0 == i1 for an odd count)."""
    n = len(x)
    return ((n - 1) // 2, (n - 1) // 2) if n % 2 else (n // 2 - 1, n // 2)


def _at_centre(f, axes_pairs):
    """Mean of f over the centre node(s) along the given (axis, (i0, i1)) pairs."""
    f = np.asarray(f, dtype=np.float64)
    for axis, (i0, i1) in axes_pairs:
        f = 0.5 * (np.take(f, i0, axis=axis) + np.take(f, i1, axis=axis))
    return float(f)


def _centre_derivative(f, x, axis, others):
    """df/dx at x* = 1/2 along `axis`: the centred difference over the two
    neighbours of the centre node (odd count: exact on quadratics on the
    symmetric mesh) or over the two centre nodes (even count), averaged over
    the centre node(s) of the other axes."""
    f = np.asarray(f, dtype=np.float64)
    i0, i1 = _centre_pair(x)
    if i0 == i1:
        a, b = i0 - 1, i0 + 1
    else:
        a, b = i0, i1
    d = (np.take(f, b, axis=axis) - np.take(f, a, axis=axis)) / (x[b] - x[a])
    pairs = [(ax if ax < axis else ax - 1, p) for ax, p in others]
    pairs.sort(key=lambda t: -t[0])
    return _at_centre(d, pairs)


def centre_values_2d(xi_x, xi_y, T, u, v):
    """T, u, v and the vorticity dv/dx - du/dy at the cavity centre x* = y* = 1/2
    (Table 3), in the units of the inputs per unit x* (fields [ny][nx]).  With an
    even node count the centre lies between nodes: values are the mean of the
    two (four) centre nodes and derivatives the difference across the centre."""
    x, y = node_positions(xi_x), node_positions(xi_y)
    px, py = _centre_pair(x), _centre_pair(y)
    c = [(1, px), (0, py)]
    return {"T": _at_centre(T, c), "u": _at_centre(u, c), "v": _at_centre(v, c),
            "omega": _centre_derivative(v, x, 1, [(0, py)]) -
            _centre_derivative(u, y, 0, [(1, px)])}


def centre_values_3d(xi_x, xi_y, xi_z, T, u, v, w):
    """T, u, v, w and the magnitude of the vorticity vector (dw/dy - dv/dz,
    du/dz - dw/dx, dv/dx - du/dy) at the centre of the cube (the 3-D
    centre-value table; fields [nz][ny][nx], derivatives per unit x*)."""
    x, y, z = node_positions(xi_x), node_positions(xi_y), node_positions(xi_z)
    px, py, pz = _centre_pair(x), _centre_pair(y), _centre_pair(z)
    c = [(2, px), (1, py), (0, pz)]
    out = {k: _at_centre(f, c) for k, f in (("T", T), ("u", u), ("v", v), ("w", w))}

    def d(f, coord, axis):
        others = [(a, p) for a, p in ((2, px), (1, py), (0, pz)) if a != axis]
        return _centre_derivative(f, coord, axis, others)

    wx = d(w, y, 1) - d(v, z, 0)
    wy = d(u, z, 0) - d(w, x, 2)
    wz = d(v, x, 2) - d(u, y, 1)
    out["omega"] = float(np.sqrt(wx * wx + wy * wy + wz * wz))
    out["omega_z"] = wz
    return out


def prolong(fields, coarse, fine):
    """Fields of a coarse mesh carried to a finer one by multilinear
    interpolation between node positions (linear extrapolation into the
    layer between the outermost coarse nodes and the walls): the initial
    state of a finer run in a grid-refinement study.  `coarse` and `fine` are
    lists of ghost-node meshes per axis (x first); fields are arrays
    [(nz,) ny, nx]."""
    from scipy.interpolate import RegularGridInterpolator
    pc = [node_positions(m) for m in reversed(coarse)]      # array axis order
    pf = [node_positions(m) for m in reversed(fine)]
    pts = np.stack(np.meshgrid(*pf, indexing="ij"), axis=-1).reshape(-1, len(pf))
    out = {}
    for k, f in fields.items():
        it = RegularGridInterpolator(pc, np.asarray(f, dtype=np.float64), method="linear",
                                     bounds_error=False, fill_value=None)
        out[k] = it(pts).reshape([len(a) for a in pf])
    return out


def band_profiles_3d(field, y_star, z_star, band=(0.4, 0.6), wy=None, wz=None):
    """x profile of a [nz][ny][nx] field averaged over the nodes with y* and z*
    both in the band (the mid-height band of the mid-depth region)."""
    f = np.asarray(field, dtype=np.float64)
    ry = (y_star >= band[0]) & (y_star <= band[1])
    rz = (z_star >= band[0]) & (z_star <= band[1])
    wy = np.ones(ry.sum()) if wy is None else np.asarray(wy)[ry]
    wz = np.ones(rz.sum()) if wz is None else np.asarray(wz)[rz]
    sub = f[np.ix_(rz, ry, np.ones(f.shape[2], bool))]
    return np.einsum("zyx,z,y->x", sub, wz, wy) / (wz.sum() * wy.sum())


def divergence_3d(u, v, w, x, y, z):
    """du/dx + dv/dy + dw/dz on the non-uniform node positions ([nz][ny][nx])."""
    return np.gradient(np.asarray(u, float), np.asarray(x, float), axis=2) + \
        np.gradient(np.asarray(v, float), np.asarray(y, float), axis=1) + \
        np.gradient(np.asarray(w, float), np.asarray(z, float), axis=0)


def divergence_pdf(div, lo=-10.0, hi=0.0, bins=50):
    """Probability density of log10 |div| over the nodes (the divergence
    histograms of Sec. 3 and Sec. 4): bin centres, densities (integrating to the
    share of nodes inside [lo, hi]) and the share of nodes below and above."""
    a = np.abs(np.asarray(div, dtype=np.float64)).ravel()
    with np.errstate(divide="ignore"):
        la = np.log10(a)
    n = a.size
    hist, edges = np.histogram(la[np.isfinite(la)], bins=bins, range=(lo, hi))
    width = (hi - lo) / bins
    return {"centres": 0.5 * (edges[1:] + edges[:-1]), "density": hist / (n * width),
            "below": float(np.sum(~np.isfinite(la) | (la < lo))) / n,
            "above": float(np.sum(la > hi)) / n,
            "median_log10": float(np.median(la[np.isfinite(la)])) if np.isfinite(la).any()
            else float("-inf")}

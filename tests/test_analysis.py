"""The grid-convergence helpers against the p, infinity and GCI rows that
Table 2 prints for its own three meshes (tests/golden/table2_*.json)."""
import json
import math
import os

import pytest

from paper_2509_01099_gb300 import analysis as A

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", ["table2_ra1e6.json", "table2_ra1e8.json"])
def test_convergence_table_reproduces_table2(name):
    data = json.load(open(os.path.join(GOLDEN, name)))
    for key, row in data.items():
        if not isinstance(row, dict) or "values" not in row:
            continue
        c, m, f = row["values"]
        got = A.convergence_table({key: (c, m, f)})[key]
        # p is printed to one decimal and computed from values rounded to 4
        # decimals: |dp| <= (|1/(c-m)| + |1/(m-f)|) * 0.5e-4 * 2 / ln 2 from that rounding
        dp = (abs(1 / (c - m)) + abs(1 / (m - f))) * 1e-4 / math.log(2)
        assert abs(got["p"] - row["p"]) <= 0.05 + dp, (key, got["p"], row["p"])
        assert abs(got["inf"] - row["inf"]) <= 2e-4 * max(1.0, abs(row["inf"]) / 10), key
        # GCI with the printed order: two significant digits
        g = A.gci_percent(m, f, row["p"])
        assert abs(g / row["gci_percent"] - 1) < 0.2, (key, g)


def test_exact_power_law_is_recovered():
    # f(h) = 3 + 0.5 h^2.5 on h = 1, 1/2, 1/4
    f = [3 + 0.5 * h ** 2.5 for h in (1.0, 0.5, 0.25)]
    t = A.convergence_table({"q": tuple(f)})["q"]
    assert abs(t["p"] - 2.5) < 1e-12 and abs(t["inf"] - 3.0) < 1e-12


def test_degenerate_rows_report_none():
    t = A.convergence_table({"flat": (1.0, 1.0, 1.0)})["flat"]
    assert t["p"] is None and t["inf"] is None


def test_boundary_layer_methods_on_closed_forms():
    # T* = 1 - (1 - Tc) (1 - exp(-x/d)) and v* = V (x/d) exp(1 - x/d): the slope
    # method recovers d for T (wall slope (1 - Tc)/d) and d for v (v_max = V at
    # x = d, wall slope V e / d -> delta_V = d / e); the 99% points are
    # d ln(100) for T and the first crossing below the maximum for v.
    import numpy as np
    d, Tc, V = 0.02, 0.5, 0.3
    x = np.linspace(0.0005, 0.5, 4000)
    T = 1 - (1 - Tc) * (1 - np.exp(-x / d))
    v = V * (x / d) * np.exp(1 - x / d)
    bl = A.boundary_layers(x, T, v)
    assert abs(bl["delta_T_slope"] - d) < 1e-3 * d
    assert abs(bl["delta_V_slope"] - d / math.e) < 1e-3 * d
    assert abs(bl["delta_T_99"] - d * math.log(100)) < 1e-3 * d
    # 99% of the maximum of s e^(1-s) on the rising side: s = 0.86484...
    assert abs(bl["delta_V_99"] - 0.864843 * d) < 2e-3 * d


def test_power_law_and_divergence():
    import numpy as np
    ra = np.array([1e6, 1e7, 1e8])
    p, c = A.power_law(ra, 3.0 * ra ** -0.25)
    assert abs(p + 0.25) < 1e-12 and abs(c - 3.0) < 1e-9
    x = np.sort(np.random.default_rng(1).uniform(0, 1, 40))
    y = np.sort(np.random.default_rng(2).uniform(0, 1, 30))
    X, Y = np.meshgrid(x, y)
    # a divergence-free field (u, v) = (x, -y) and one with divergence 2: (x, y)
    assert np.abs(A.divergence_2d(X, -Y, x, y)).max() < 1e-12
    assert np.abs(A.divergence_2d(X, Y, x, y) - 2).max() < 1e-12
    # node positions of the uniform mesh: cell centres
    from oracle import islbm_oracle as O
    np.testing.assert_allclose(A.node_positions(O.mesh_uniform(8)), (np.arange(8) + 0.5) / 8,
                               rtol=0, atol=1e-15)


def _mesh_xy(kind, n):
    from oracle import islbm_oracle as O
    return O.mesh_erf(n, 1.5) if kind == "erf" else O.mesh_uniform(n)


@pytest.mark.parametrize("n", [17, 16])
def test_centre_values_2d_on_closed_forms(n):
    """Linear and quadratic fields about the centre: the centre values and the
    vorticity dv/dx - du/dy are exact (odd n: the centre node; even n: the mean
    of the centre nodes and the difference across the centre, both exact for
    fields symmetric in their quadratic part)."""
    import numpy as np
    xi = _mesh_xy("erf", n)
    x = A.node_positions(xi)
    X, Y = np.meshgrid(x, x)
    a, b = 0.7, -1.3
    u = a * (Y - 0.5) + 0.2
    v = b * (X - 0.5) - 0.1 + 3 * (Y - 0.5) ** 2
    T = 0.5 + 0.3 * (X - 0.5) + 2 * (X - 0.5) ** 2 * 0
    c = A.centre_values_2d(xi, xi, T, u, v)
    assert abs(c["omega"] - (b - a)) < 1e-12
    assert abs(c["u"] - 0.2) < 1e-12 and abs(c["T"] - 0.5) < 1e-12
    expect_v = -0.1 + (0.0 if n % 2 else 3 * (x[n // 2] - 0.5) ** 2)
    assert abs(c["v"] - expect_v) < 1e-12
    # rigid rotation (u, v) = (-(y - 1/2), x - 1/2): vorticity 2
    assert abs(A.centre_values_2d(xi, xi, T, -(Y - 0.5), X - 0.5)["omega"] - 2) < 1e-12


def test_centre_values_3d_and_band_profiles_3d():
    import numpy as np
    xi_x, xi_y, xi_z = _mesh_xy("erf", 9), _mesh_xy("uniform", 10), _mesh_xy("erf", 11)
    x, y, z = (A.node_positions(m) for m in (xi_x, xi_y, xi_z))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    T = 0.5 + (X - 0.5) * (Y - 0.5) + 0.1 * (Z - 0.5)
    c = A.centre_values_3d(xi_x, xi_y, xi_z, T, X - 0.5, 2 * (Y - 0.5), 0.3 + 0 * Z)
    assert abs(c["T"] - 0.5) < 1e-12 and abs(c["u"]) < 1e-12
    assert abs(c["v"]) < 1e-12 and abs(c["w"] - 0.3) < 1e-12
    # a field that depends on x only: the band profile is the field itself
    prof = A.band_profiles_3d(np.sin(3 * X), y, z)
    np.testing.assert_allclose(prof, np.sin(3 * x), rtol=0, atol=1e-14)
    # separable weights: the average of g(y) h(z) over the band is the product of averages
    g = np.cos(Y) * np.exp(Z)
    prof = A.band_profiles_3d(g, y, z)
    band_y = (y >= 0.4) & (y <= 0.6)
    band_z = (z >= 0.4) & (z <= 0.6)
    expect = np.cos(y[band_y]).mean() * np.exp(z[band_z]).mean()
    np.testing.assert_allclose(prof, expect, rtol=1e-13)


def test_divergence_3d_and_its_pdf():
    import numpy as np
    rng = np.random.default_rng(3)
    x, y, z = (np.sort(rng.uniform(0, 1, n)) for n in (12, 9, 7))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    assert np.abs(A.divergence_3d(X, Y, -2 * Z, x, y, z)).max() < 1e-12
    assert np.abs(A.divergence_3d(X, Y, Z, x, y, z) - 3).max() < 1e-12
    # |div| log-uniform over [1e-8, 1e-2]: a flat density of 1/6 per decade there
    d = 10 ** rng.uniform(-8, -2, 200_000) * rng.choice([-1, 1], 200_000)
    pdf = A.divergence_pdf(d, lo=-10, hi=0, bins=20)
    inside = (pdf["centres"] > -8) & (pdf["centres"] < -2)
    np.testing.assert_allclose(pdf["density"][inside], 1 / 6, rtol=0.03)
    assert np.all(pdf["density"][~inside] == 0)
    assert abs(pdf["density"].sum() * 0.5 - 1) < 1e-12 and pdf["below"] == 0 == pdf["above"]
    assert abs(pdf["median_log10"] + 5) < 0.02
    zero = A.divergence_pdf(np.zeros(10))
    assert zero["below"] == 1.0


def test_centre_vorticity_3d_of_rigid_rotations():
    import numpy as np
    xi_x, xi_y, xi_z = _mesh_xy("erf", 9), _mesh_xy("uniform", 10), _mesh_xy("erf", 11)
    x, y, z = (A.node_positions(m) for m in (xi_x, xi_y, xi_z))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    T = 0 * X
    # rotation about z: (u, v, w) = (-(y-1/2), x-1/2, 0): vorticity (0, 0, 2)
    c = A.centre_values_3d(xi_x, xi_y, xi_z, T, -(Y - 0.5), X - 0.5, 0 * X)
    assert abs(c["omega"] - 2) < 1e-12 and abs(c["omega_z"] - 2) < 1e-12
    # rotation about x with rate 3: (0, -3(z-1/2), 3(y-1/2)): vorticity (6, 0, 0)
    c = A.centre_values_3d(xi_x, xi_y, xi_z, T, 0 * X, -3 * (Z - 0.5), 3 * (Y - 0.5))
    assert abs(c["omega"] - 6) < 1e-12 and abs(c["omega_z"]) < 1e-12


def test_prolong_is_exact_on_linear_fields():
    import numpy as np
    from oracle import islbm_oracle as O
    coarse = [O.mesh_erf(9, 1.5), O.mesh_erf(7, 1.5)]
    fine = [O.mesh_erf(17, 1.5), O.mesh_erf(13, 1.5)]
    xc, yc = A.node_positions(coarse[0]), A.node_positions(coarse[1])
    xf, yf = A.node_positions(fine[0]), A.node_positions(fine[1])
    Yc, Xc = np.meshgrid(yc, xc, indexing="ij")
    Yf, Xf = np.meshgrid(yf, xf, indexing="ij")
    out = A.prolong({"T": 0.3 + 2 * Xc - Yc}, coarse, fine)
    np.testing.assert_allclose(out["T"], 0.3 + 2 * Xf - Yf, atol=1e-13)
    # 3-D, with extrapolation into the wall layers
    c3 = [O.mesh_erf(5, 1.5)] * 3
    f3 = [O.mesh_erf(9, 1.5)] * 3
    p = A.node_positions(c3[0])
    q = A.node_positions(f3[0])
    Z, Y, X = np.meshgrid(p, p, p, indexing="ij")
    Zf, Yf, Xf = np.meshgrid(q, q, q, indexing="ij")
    out = A.prolong({"u": X + 2 * Y + 3 * Z}, c3, f3)
    np.testing.assert_allclose(out["u"], Xf + 2 * Yf + 3 * Zf, atol=1e-12)

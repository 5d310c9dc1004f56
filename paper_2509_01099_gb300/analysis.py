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

"""Tile order of the 2-D TMA step where tiles are claimed from a device counter.

On a 2048^2 mesh the step has 8,192 tiles of 64 x 8 nodes for at most 304
resident CTAs (152 SMs x 2), more than the 24 tiles per CTA from which the
launch hands tiles out by a counter instead of a fixed stride.  A tile that is
skipped, a tile computed from another tile's staged data, or a counter left
unreset between launches (the last CTA resets it) shows up as an O(1) error:
the stale buffer holds the state of two steps earlier.
"""
import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import random_populations, random_signed, temperature_noise
from tests.helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA device")]

N = 2048


def _pkg():
    from paper_2509_01099_gb300 import build as B
    B.build()
    import paper_2509_01099_gb300 as pkg
    return pkg


def test_claimed_tiles_every_population_against_oracle():
    """Three steps from a far-from-equilibrium random state: all 58.7M
    populations against the FP64 oracle at the FP32 population tolerance."""
    pkg = _pkg()
    xi = O.mesh_tanh(N, 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e8))
    f = random_populations(9, cav.shape, seed=31, spread=0.2)
    g = random_signed(5, cav.shape, seed=32, amplitude=0.12)
    cav.init_populations(f, g)
    cav.step(3)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(xi, xi, Ra=1e8, precision="fp32", kernel="tma_r2s2")
    s.set_populations(f, g)
    s.step(3)
    fp, gp = s.populations()
    s.close()
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= 2e-6
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= 2e-6


def test_claimed_tiles_over_many_launches_match_one_tile_per_cta():
    """70 steps (a captured graph of 64 launches, then 6 single launches) of the
    claimed order against the kernel that stages one tile per CTA with no tile
    order at all: the same arithmetic per node, so the fields agree to FP32
    rounding."""
    pkg = _pkg()
    xi = pkg.islbm_mesh_tanh(N, 1.5)
    out = {}
    for kernel in ("tma_r2s2", "tiled"):
        s = pkg.Solver(xi, xi, Ra=1e8, precision="fp32", kernel=kernel)
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=4))
        s.step(70)
        out[kernel] = s.fields()
        assert s.reduce()["status"] == 0
        s.close()
    for k in ("T", "u", "v"):
        a, b = out["tma_r2s2"][k], out["tiled"][k]
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k

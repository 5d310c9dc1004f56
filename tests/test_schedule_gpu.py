"""Tile order of the 2-D TMA step where tiles are claimed from a device counter.

On a 2048^2 mesh the step has 8,192 tiles of 64 x 8 nodes for at most 304
resident CTAs (152 SMs x 2): 26 per CTA, which the launch hands out at a fixed
stride by default.  ISLBM_TMA_SCHEDULE=claimed claims every tile after the
first two from a counter (the default from 64 tiles per CTA), and
ISLBM_TMA_SCHEDULE=tail takes the first 25 at the fixed stride and claims the
rest.  A
tile that is skipped, a tile computed from another tile's staged data, or a
counter left unreset between launches (the last CTA resets it) shows up as an
O(1) error: the stale buffer holds the state of two steps earlier.
"""
import json
import os
import subprocess
import sys

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


def test_default_tile_order_every_population_against_oracle():
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


_SUBPROCESS = r"""
import json, sys
import numpy as np
import paper_2509_01099_gb300 as pkg
from synthetic import temperature_noise
xi = pkg.islbm_mesh_tanh(%d, 1.5)
out = {}
for kernel in ("tma_r2s2", "tiled"):
    s = pkg.Solver(xi, xi, Ra=1e8, precision="fp32", kernel=kernel)
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=4))
    s.step(70)
    out[kernel] = s.fields()
    assert s.reduce()["status"] == 0
    s.close()
err = {k: float(np.abs(out["tma_r2s2"][k] - out["tiled"][k]).max() / np.abs(out["tiled"][k]).max())
       for k in ("T", "u", "v")}
print(json.dumps(err))
"""


@pytest.mark.parametrize("schedule", ["default", "claimed", "tail"])
def test_tile_orders_over_many_launches_match_one_tile_per_cta(schedule):
    """70 steps (a captured graph of 64 launches, then 6 single launches) in
    each tile order against the kernel that stages one tile per CTA with no
    tile order at all: the same arithmetic per node, so the fields agree to
    FP32 rounding.  The order is read once per process, so each runs in a
    process of its own."""
    _pkg()
    env = dict(os.environ)
    env.pop("ISLBM_TMA_SCHEDULE", None)
    if schedule != "default":
        env["ISLBM_TMA_SCHEDULE"] = schedule
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _SUBPROCESS % N], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    err = json.loads(r.stdout.strip().splitlines()[-1])
    for k, e in err.items():
        assert e <= 1e-6, (schedule, k, e)

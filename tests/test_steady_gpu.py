"""Steady-state criterion on the GPU (Sec. 3) against the oracle's, through the C ABI."""
import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import temperature_noise
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("d", [2, 3])
def test_steady_change_matches_the_oracle(d):
    n = 40 if d == 2 else 12
    xi = O.mesh_tanh(n, 1.5)
    meshes = (xi, xi) if d == 2 else (xi, xi, xi)
    cav = O.Cavity(*meshes, params=O.Params(Ra=1e6))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=4))
    cav.step(500)
    _, u0, T0 = cav.fields()
    cav.step(200)
    _, u1, T1 = cav.fields()
    Ts = lambda T: T - cav.T0            # T* with dT = 1
    ref = O.steady_change(u1, u0, Ts(T1), Ts(T0))
    s = pkg.Solver(*meshes, Ra=1e6, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=4))
    assert s.steady_change() == (np.inf, np.inf)          # first call: snapshot only
    s.step(500)
    s.steady_change()
    s.step(200)
    du, dT = s.steady_change()
    s.close()
    assert abs(du / ref[0] - 1) < 1e-9 and abs(dT / ref[1] - 1) < 1e-9, (du, dT, ref)


def test_run_to_steady_and_budget():
    xi = O.mesh_erf(24, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e4, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    r = s.run_to_steady(tol=1e-3, interval=200, max_steps=400, check=False)
    assert r["status"] == 5 and r["steps"] == 400                 # ISLBM_ERR_NOT_CONVERGED
    r = s.run_to_steady(tol=1e-9, interval=2000, max_steps=2_000_000)
    assert r["du"] < 1e-9 and r["dT"] < 1e-9 and r["steps"] % 2000 == 0
    a = s.reduce()
    s.step(4000)
    b = s.reduce()
    assert abs(a["Nu"] / b["Nu"] - 1) < 1e-8
    s.close()

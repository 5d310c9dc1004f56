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


@pytest.mark.parametrize("dim", [2, 3])
def test_time_average_accumulators(dim):
    """The FP64 accumulators return the mean of the states added, and reset."""
    xi = O.mesh_tanh(10, 1.5)
    s = pkg.Solver(*([xi] * dim), Ra=1e6, precision="fp32")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=1))
    with pytest.raises(pkg.IslbmError):
        s.average()                       # nothing accumulated yet
    keys = ("T", "u", "v") + (("w",) if dim == 3 else ())
    snaps = []
    s.average_reset()
    for _ in range(3):
        s.step(37)
        s.average_add()
        f = s.fields()
        snaps.append({k: f[k] for k in keys})
    mean, count = s.average()
    assert count == 3
    for k in keys:
        ref = (snaps[0][k] + snaps[1][k] + snaps[2][k]) / 3
        assert np.abs(mean[k] - ref).max() <= 1e-15 * max(np.abs(ref).max(), 1e-300) * 4
    s.average_reset()
    s.average_add()
    mean, count = s.average()
    f = s.fields()
    assert count == 1 and np.array_equal(mean["T"], f["T"])
    s.close()

"""Batched cavities (one persistent launch over many cavities of different sizes)
and the tile-shape autotuner."""
import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import ra_sweep, temperature_noise
from tests.helpers import gpu_available, rel_field_error

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

CAVS = [dict(n=48, mesh="tanh", Ra=1e6), dict(n=64, mesh="erf", Ra=3e6),
        dict(n=45, mesh="uniform", Ra=1e5), dict(n=80, mesh="tanh", Ra=1e7)]


def _xi(c):
    return (pkg.islbm_mesh_uniform(c["n"]) if c["mesh"] == "uniform"
            else getattr(pkg, "islbm_mesh_" + c["mesh"])(c["n"], 1.5))


def test_batch_members_equal_single_solvers_bitwise():
    b = pkg.Batch(CAVS, precision="fp32")
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    b.step(64 + 64 + 9)                    # graph replays + single launches
    b.synchronize()
    for k, (c, m) in enumerate(zip(CAVS, b.members)):
        rows = b.tile_rows(k)
        kern = "tma_r2s2" if rows == 8 else "tma_r4s2"
        s = pkg.Solver(_xi(c), _xi(c), Ra=c["Ra"], precision="fp32", kernel=kern)
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=k))
        s.step(137)
        fa, ga = m.populations()
        fb, gb = s.populations()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ga, gb)
        assert m.time == 137
        s.close()
    b.close()


def test_batch_member_against_the_oracle():
    b = pkg.Batch(CAVS[:2], precision="fp32")
    c = CAVS[1]
    m = b.members[1]
    m.set_fields(temperature_noise(m.shape, 1e-6, seed=3))
    b.members[0].set_fields(temperature_noise(b.members[0].shape, 1e-6, seed=4))
    b.step(500)
    got = m.fields()
    xi = O.mesh_erf(c["n"], 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=c["Ra"]))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=3))
    cav.step(500)
    rho, u, T = cav.fields()
    assert rel_field_error(got["T"], T) < 1e-5
    assert rel_field_error(got["v"], u[1]) < 1e-5
    b.close()


def test_autotune_picks_a_runnable_variant():
    best, us = pkg.islbm_autotune(128, "tanh", 1.5, "fp32")
    assert 1 <= best <= 6 and np.isfinite(us[best]) and us[best] == min(us[1:])
    best2, us2 = pkg.islbm_autotune(128, "tanh", 1.5, "fp32")   # cached
    assert best2 == best and us2 == us


def test_autotuned_sweep_batch_runs_to_steady():
    ra, n = ra_sweep(6, seed=0, log10_lo=3.0, log10_hi=4.0, sizes=(24, 32, 40))
    cavs = [dict(n=int(k), mesh="tanh", Ra=float(r)) for r, k in zip(ra, n)]
    b = pkg.Batch(cavs, precision="fp32", autotune=True)
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    steps, st = b.run_to_steady(tol=1e-6, interval=1000, max_steps=400_000)
    assert st == 0 and all(s > 0 for s in steps)
    for m in b.members:
        r = m.reduce()
        assert 1.0 < r["Nu"] < 3.0
    b.close()


def test_batch_steady_nu_criterion():
    """Window means of Nu: the reported step count is a whole number of windows,
    the reported mean agrees with the Nu the field criterion converges to, and
    the arguments are validated."""
    cavs = [dict(n=32, mesh="tanh", Ra=1e4), dict(n=40, mesh="tanh", Ra=3e4)]
    b = pkg.Batch(cavs, precision="fp32")
    with pytest.raises(pkg.IslbmError):
        b.run_to_steady_nu(tol=0.0)
    with pytest.raises(pkg.IslbmError):
        b.run_to_steady_nu(window=1)
    steps, nu, re, st = b.run_to_steady_nu(tol=1e-4, sample=200, window=20, max_steps=400_000)
    assert st == 0
    for s in steps:
        assert s > 0 and s % (200 * 20) == 0
    ref = pkg.Batch(cavs, precision="fp32")
    ref.run_to_steady(tol=1e-6, interval=1000, max_steps=600_000)
    for k, m in enumerate(ref.members):
        r = m.reduce()
        assert abs(nu[k] - r["Nu"]) < 2e-3 * r["Nu"]
        assert abs(re[k] - r["Re"]) < 5e-3 * r["Re"]
    # a budget shorter than two windows cannot converge
    c = pkg.Batch(cavs, precision="fp32")
    steps, nu, re, st = c.run_to_steady_nu(tol=1e-4, sample=100, window=10, max_steps=1500,
                                           check=False)
    assert st == 5 and steps == [-1, -1]      # ISLBM_ERR_NOT_CONVERGED
    for x in (b, ref, c):
        x.close()


def test_batch_retires_converged_cavities_and_resumes_them():
    """A cavity that has met the criterion leaves the work list (no further
    steps are spent on it); when the call returns every cavity is advanced
    again, and each equals a single solver that took as many steps."""
    cavs = [dict(n=24, mesh="tanh", Ra=1e3), dict(n=40, mesh="tanh", Ra=3e4)]
    b = pkg.Batch(cavs, precision="fp32")
    steps, nu, re, st = b.run_to_steady_nu(tol=1e-4, sample=200, window=10, max_steps=600_000)
    assert st == 0 and steps[0] < steps[1]
    infos = [pkg.islbm_info(m.h) for m in b.members]
    assert infos[0].time == steps[0] and infos[1].time == steps[1]
    # every cavity steps again after the call: each equals a single solver that
    # took the same number of steps from the same (rest) state, bitwise
    b.step(70)
    b.synchronize()
    for k, (m, c) in enumerate(zip(b.members, cavs)):
        s = pkg.Solver(pkg.islbm_mesh_tanh(c["n"], 1.5), pkg.islbm_mesh_tanh(c["n"], 1.5),
                       Ra=c["Ra"], precision="fp32", kernel="tma_r2s2")
        s.step(steps[k] + 70)
        ref = s.fields()
        got = m.fields()
        for key in ("T", "u", "v"):
            assert np.array_equal(got[key], ref[key]), (k, key)
        s.close()
    b.close()

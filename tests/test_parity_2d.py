"""GPU parity of the 2-D CUDA path against the FP64 oracle, through the C ABI.

Tolerances (field-relative error max|gpu - oracle| / max|oracle|):
  FP64 storage:  1e-11 on T, u, v; Nu/Re to 1e-10 relative.  Both sides round at
                 1e-16 relative per operation, in different orders, on O(0.1)
                 populations; early in a run |u| is ~1e-3 of them, so the
                 field-relative error of u carries a ~1e3 amplification and
                 grows like the square root of the step count (measured:
                 2.6e-12 after 200 steps).
  FP32 storage:  1e-5 on T, u, v after 1000 steps; Nu within 1e-4 relative.
  FP16/BF16 deviation storage: errors are reported against loose sanity bounds
  (the target for them is the steady Nu, checked elsewhere).
"""
import functools
import os
import tempfile

import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import random_populations, random_signed, temperature_noise
from tests.helpers import gpu_available, rel_field_error, rel_vector_error

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

MESHES = {
    "tanh64": lambda: (O.mesh_tanh(64, 1.5), O.mesh_tanh(64, 1.5)),
    "uniform64": lambda: (O.mesh_uniform(64), O.mesh_uniform(64)),
    "erf45": lambda: (O.mesh_erf(45, 1.5), O.mesh_erf(45, 1.5)),
    # rectangular ragged cavity: 37 x 29 nodes of one lattice unit (x extent 37/29 H)
    "uniform37x29": lambda: ((np.arange(39) - 0.5) / 29, O.mesh_uniform(29)),
}


@functools.lru_cache(maxsize=None)
def oracle_run(mesh: str, Ra: float, steps: int, stencil: str = "centred"):
    xi_x, xi_y = MESHES[mesh]()
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=Ra, stencil=stencil))
    T0 = temperature_noise(cav.shape, 1e-6, seed=0)
    cav.init_fields(T0)
    cav.step(steps)
    rho, u, T = cav.fields()
    return {"rho": rho, "u": u[0], "v": u[1], "T": T, "red": cav.reductions(), "T_init": T0}


def gpu_run(mesh, Ra, steps, precision, stencil="centred"):
    xi_x, xi_y = MESHES[mesh]()
    s = pkg.Solver(xi_x, xi_y, Ra=Ra, precision=precision, stencil=stencil)
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(steps)
    out = s.fields()
    out["red"] = s.reduce()
    s.close()
    return out


TOL = {"fp64": 1e-11, "fp32": 1e-5}
NU_TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_cavity_fields_after_1000_steps(mesh, precision):
    ref = oracle_run(mesh, 1e6, 1000)
    got = gpu_run(mesh, 1e6, 1000, precision)
    assert rel_field_error(got["T"], ref["T"]) <= TOL[precision]
    err_u = rel_vector_error([got["u"], got["v"]], [ref["u"], ref["v"]])
    assert err_u <= TOL[precision], err_u
    for k in ("u", "v"):   # each component on its own scale as well (2-D: similar sizes)
        assert rel_field_error(got[k], ref[k]) <= 3 * TOL[precision], k
    assert np.abs(got["rho"] - ref["rho"]).max() <= 10 * TOL[precision]
    for k in ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re"):
        # Nusselt numbers are O(1) (conduction: 1); early in a run Nu_middle is
        # near zero, so the bound is taken on that scale
        r = abs(got["red"][k] - ref["red"][k]) / max(1.0, abs(ref["red"][k]))
        assert r <= NU_TOL[precision], (k, got["red"][k], ref["red"][k])
    assert abs(got["red"]["mass"] / ref["red"]["mass"] - 1) <= NU_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_upwind_stencil(precision):
    ref = oracle_run("erf45", 1e6, 300, "upwind")
    got = gpu_run("erf45", 1e6, 300, precision, "upwind")
    for k in ("T", "u", "v"):
        assert rel_field_error(got[k], ref[k]) <= TOL[precision], k


def _random_state(q_f, q_g, shape, seed):
    f = random_populations(q_f, shape, seed=seed, spread=0.2)
    g = random_signed(q_g, shape, seed=seed + 1, amplitude=0.12)
    return f, g


# 16-bit stores round stochastically (error up to one ulp: 2^-10 FP16, 2^-7 BF16
# of the stored deviation per step)
POP_TOL = {"fp64": 1e-13, "fp32": 2e-6, "fp16dev": 5e-3, "bf16dev": 5e-2}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("mesh", ["erf45", "uniform37x29", "tanh64"])
@pytest.mark.parametrize("steps", [0, 1, 3])
def test_random_state_populations(mesh, precision, steps):
    """Far-from-equilibrium random populations: every population of every node after
    0 (collision only), 1 and 3 steps, element by element."""
    xi_x, xi_y = MESHES[mesh]()
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=1e6))
    f, g = _random_state(9, 5, cav.shape, seed=11)
    cav.init_populations(f, g)
    cav.step(steps)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision=precision)
    s.set_populations(f, g)
    s.step(steps)
    fp, gp = s.populations()
    s.close()
    scale_f = np.abs(fp_ref).max()
    scale_g = np.abs(gp_ref).max()
    assert np.abs(fp - fp_ref).max() / scale_f <= POP_TOL[precision]
    assert np.abs(gp - gp_ref).max() / scale_g <= POP_TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_full_size_1024_tanh_one_step(precision):
    """The bench configuration (1024^2 tanh-stretched mesh, a = 1.5) with the same
    launch shape as the bench: two steps from a random state, all 14.7M values."""
    xi = O.mesh_tanh(1024, 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e8))
    f, g = _random_state(9, 5, cav.shape, seed=5)
    cav.init_populations(f, g)
    cav.step(2)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(xi, xi, Ra=1e8, precision=precision)
    s.set_populations(f, g)
    s.step(2)
    fp, gp = s.populations()
    s.close()
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= POP_TOL[precision]
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= POP_TOL[precision]


def test_minimum_size_and_odd_centre():
    for n in (4, 5):
        xi = O.mesh_erf(n, 1.5)
        cav = O.Cavity(xi, xi, params=O.Params(Ra=1e3))
        cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=3))
        cav.step(50)
        s = pkg.Solver(xi, xi, Ra=1e3, precision="fp64")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=3))
        s.step(50)
        got, red = s.fields(), s.reduce()
        s.close()
        rho, u, T = cav.fields()
        assert rel_field_error(got["T"], T) < 1e-11
        ref = cav.reductions()
        for k in ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re"):
            assert abs(red[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), (n, k)


def test_uniform_mesh_is_detected():
    s = pkg.Solver(O.mesh_uniform(32), O.mesh_uniform(32), Ra=1e5, precision="fp32")
    assert s.info.uniform == 1
    s.close()
    s = pkg.Solver(O.mesh_tanh(32, 1.5), O.mesh_tanh(32, 1.5), Ra=1e5, precision="fp32")
    assert s.info.uniform == 0
    s.close()


def test_checkpoint_roundtrip_is_bitwise():
    xi = O.mesh_tanh(48, 1.5)
    a = pkg.Solver(xi, xi, Ra=1e6, precision="fp32")
    a.set_fields(temperature_noise(a.shape, 1e-6, seed=0))
    a.step(200)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        a.step(200)
        fa, ga = a.populations()
        b = pkg.Solver(xi, xi, Ra=1e6, precision="fp32")
        b.load(path)
        assert b.time == 200
        b.step(200)
        fb, gb = b.populations()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ga, gb)
        c = pkg.Solver(xi, xi, Ra=1e7, precision="fp32")     # other configuration
        with pytest.raises(pkg.IslbmError) as e:
            c.load(path)
        assert e.value.status == 7
        with open(path, "r+b") as fh:                          # truncated file
            fh.truncate(1000)
        with pytest.raises(pkg.IslbmError) as e:
            b.load(path)
        assert e.value.status == 7
        for s in (a, b, c):
            s.close()


def test_nonfinite_state_is_reported():
    xi = O.mesh_erf(16, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e6, precision="fp32")
    T = np.zeros(s.shape)
    T[5, 7] = np.nan
    s.set_fields(T)
    s.step(3)
    r = s.reduce(check=False)
    assert r["status"] == 4 and r["nonfinite"] > 0
    with pytest.raises(pkg.IslbmError):
        s.reduce()
    s.close()


def test_step_counter_and_zero_steps():
    xi = O.mesh_erf(16, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e6, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=1))
    f0, g0 = s.populations()
    s.step(0)
    f1, g1 = s.populations()
    np.testing.assert_array_equal(f0, f1)
    s.step(7)
    assert s.time == 7
    with pytest.raises(pkg.IslbmError):
        s.step(-1)
    s.close()


VARIANTS = ["direct", "tiled", "tma_r4s2", "tma_r2s2", "tma_r2s3", "tma_r4s3"]


@pytest.mark.parametrize("kernel", VARIANTS)
@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("mesh", ["erf45", "uniform37x29", "tanh64"])
def test_every_kernel_variant_random_state(mesh, precision, kernel):
    """Each step-kernel variant, on ragged and tile-aligned meshes, from a random
    state: every population after 3 steps."""
    xi_x, xi_y = MESHES[mesh]()
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=1e6))
    f, g = _random_state(9, 5, cav.shape, seed=13)
    cav.init_populations(f, g)
    cav.step(3)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision=precision, kernel=kernel)
    assert s.info.kernel == pkg.KERNELS[kernel]
    s.set_populations(f, g)
    s.step(3)
    s.synchronize()
    fp, gp = s.populations()
    s.close()
    tol = {"fp32": 5e-6, "fp16dev": 5e-3, "bf16dev": 5e-2}[precision]
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= tol
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= tol


@pytest.mark.parametrize("kernel", VARIANTS)
def test_every_kernel_variant_cavity(kernel):
    ref = oracle_run("tanh64", 1e6, 1000)
    xi_x, xi_y = MESHES["tanh64"]()
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision="fp32", kernel=kernel)
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(1000)
    got = s.fields()
    red = s.reduce()
    s.close()
    assert rel_field_error(got["T"], ref["T"]) <= 1e-5
    assert rel_vector_error([got["u"], got["v"]], [ref["u"], ref["v"]]) <= 1e-5
    assert abs(red["Nu"] / ref["red"]["Nu"] - 1) <= 1e-4


def test_default_kernel_choice():
    s = pkg.Solver(O.mesh_tanh(64, 1.5), O.mesh_tanh(64, 1.5), Ra=1e6, precision="fp32")
    assert s.info.kernel >= 3          # pipelined TMA kernel on a stretched mesh
    s.close()
    s = pkg.Solver(O.mesh_uniform(64), O.mesh_uniform(64), Ra=1e6, precision="fp32")
    assert s.info.kernel == 1
    s.close()
    s = pkg.Solver(O.mesh_tanh(64, 1.5), O.mesh_tanh(64, 1.5), Ra=1e6, precision="fp64")
    assert s.info.kernel == 1
    s.close()


@pytest.mark.parametrize("kernel", ["direct", "tma_r2s2"])
def test_graph_replay_is_bitwise_identical(kernel):
    """islbm_step replays blocks of 64 steps from a captured CUDA graph; the result
    equals 64 + 64 + 7 single launches bit for bit, for both buffer parities."""
    xi = O.mesh_tanh(48, 1.5)
    states = []
    for chunks in ([135], [1] * 135):
        s = pkg.Solver(xi, xi, Ra=1e6, precision="fp32", kernel=kernel)
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=6))
        s.step(7)                       # start the graphs from the other buffer too
        for c in chunks:
            s.step(c)
        s.synchronize()
        states.append(s.populations())
        assert s.time == 142
        s.close()
    np.testing.assert_array_equal(states[0][0], states[1][0])
    np.testing.assert_array_equal(states[0][1], states[1][1])

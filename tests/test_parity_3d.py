"""GPU parity of the 3-D CUDA path (D3Q19 + D3Q7) against the FP64 oracle.

Tolerances as in the 2-D tests: 1e-11 (FP64) and 1e-5 (FP32) relative to the
field's largest value, with the velocity measured as one vector field (the
spanwise component w is ~1e-2 of u early in a run, so normalising it by
itself would amplify rounding by 1e2).  Far-from-equilibrium population
states accumulate about 3 steps x 50 operations of rounding: bounds 1e-13
(FP64), 5e-6 (FP32, unit roundoff 6e-8), 5e-3 (FP16 storage of deviations,
2^-11 relative) and 5e-2 (BF16 storage, 2^-8 relative), relative to the
largest population.
"""
import functools

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
    "erf14": lambda: (O.mesh_erf(14, 1.5),) * 3,
    "tanh16": lambda: (O.mesh_tanh(16, 1.5),) * 3,
    # ragged box of unit spacings: 11 x 9 x 7 nodes (height 9)
    "uniform11x9x7": lambda: ((np.arange(13) - 0.5) / 9, O.mesh_uniform(9),
                              (np.arange(9) - 0.5) / 9),
}
TOL = {"fp64": 1e-11, "fp32": 1e-5}
NU_TOL = {"fp64": 1e-10, "fp32": 1e-4}


@functools.lru_cache(maxsize=None)
def oracle_run(mesh, Ra, steps):
    xi = MESHES[mesh]()
    cav = O.Cavity(*xi, params=O.Params(Ra=Ra))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(steps)
    rho, u, T = cav.fields()
    return {"rho": rho, "u": u[0], "v": u[1], "w": u[2], "T": T, "red": cav.reductions()}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_cavity_fields_3d(mesh, precision):
    steps = 1000
    ref = oracle_run(mesh, 1e6, steps)
    xi = MESHES[mesh]()
    s = pkg.Solver(*xi, Ra=1e6, precision=precision)
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(steps)
    got = s.fields()
    red = s.reduce()
    s.close()
    assert rel_field_error(got["T"], ref["T"]) <= TOL[precision]
    err_u = rel_vector_error([got[k] for k in "uvw"], [ref[k] for k in "uvw"])
    assert err_u <= TOL[precision], err_u
    for k in ("Nu", "Nu_hot", "Nu_cold", "Re", "Re_uv"):
        r = abs(red[k] - ref["red"][k]) / max(1.0, abs(ref["red"][k]))
        assert r <= NU_TOL[precision], (k, red[k], ref["red"][k])
    assert np.isnan(red["Nu_middle"])


POP_TOL = {"fp64": 1e-13, "fp32": 5e-6, "fp16dev": 5e-3, "bf16dev": 5e-2}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("mesh", ["erf14", "uniform11x9x7"])
@pytest.mark.parametrize("steps", [0, 1, 3])
def test_random_state_populations_3d(mesh, precision, steps):
    xi = MESHES[mesh]()
    cav = O.Cavity(*xi, params=O.Params(Ra=1e6))
    f = random_populations(19, cav.shape, seed=21, spread=0.2)
    g = random_signed(7, cav.shape, seed=22, amplitude=0.08)
    cav.init_populations(f, g)
    cav.step(steps)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(*xi, Ra=1e6, precision=precision)
    s.set_populations(f, g)
    s.step(steps)
    fp, gp = s.populations()
    s.close()
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= POP_TOL[precision]
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= POP_TOL[precision]


MESHES["erf36"] = lambda: (O.mesh_erf(36, 1.5),) * 3


@pytest.mark.parametrize("kernel", ["direct", "tma3d"])
@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
def test_step_kernels_3d_random_state(kernel, precision):
    """Both 3-D step kernels on a mesh of several tiles in every direction
    (36 = 32 + a ragged 4 in x) from a far-from-equilibrium state."""
    xi = MESHES["erf36"]()
    cav = O.Cavity(*xi, params=O.Params(Ra=1e6))
    f = random_populations(19, cav.shape, seed=31, spread=0.2)
    g = random_signed(7, cav.shape, seed=32, amplitude=0.08)
    cav.init_populations(f, g)
    cav.step(3)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(*xi, Ra=1e6, precision=precision, kernel=kernel)
    assert s.info.kernel == pkg.KERNELS[kernel]
    s.set_populations(f, g)
    s.step(3)
    fp, gp = s.populations()
    s.close()
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= POP_TOL[precision]
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= POP_TOL[precision]


@functools.lru_cache(maxsize=None)
def oracle_erf36(steps):
    return oracle_run("erf36", 1e6, steps)


def test_tma3d_cavity_fields_multi_tile():
    steps = 300
    ref = oracle_erf36(steps)
    xi = MESHES["erf36"]()
    s = pkg.Solver(*xi, Ra=1e6, precision="fp32", kernel="tma3d")
    assert s.info.kernel == pkg.KERNELS["tma3d"]
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(steps)
    got = s.fields()
    red = s.reduce()
    s.close()
    assert rel_field_error(got["T"], ref["T"]) <= TOL["fp32"]
    assert rel_vector_error([got[k] for k in "uvw"], [ref[k] for k in "uvw"]) <= TOL["fp32"]
    for k in ("Nu", "Nu_hot", "Nu_cold", "Re"):
        assert abs(red[k] - ref["red"][k]) / max(1.0, abs(ref["red"][k])) <= NU_TOL["fp32"]


def test_tma3d_matches_direct_kernel_closely():
    """The two kernels apply the same operations in the same order; after 200
    steps their fields agree far inside the oracle tolerance."""
    xi = MESHES["erf36"]()
    out = {}
    for kernel in ("direct", "tma3d"):
        s = pkg.Solver(*xi, Ra=1e7, precision="fp32", kernel=kernel)
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=3))
        s.step(200)
        out[kernel] = s.fields()
        s.close()
    for k in ("T", "u", "v", "w"):
        a, b = out["direct"][k], out["tma3d"][k]
        assert np.abs(a - b).max() <= 1e-6 * max(np.abs(b).max(), 1e-30), k


def test_3d_kernel_default_choice():
    xi = O.mesh_tanh(16, 1.5)
    cases = [((xi,) * 3, "fp32", "zm3d"), ((xi,) * 3, "bf16dev", "zm3d"),
             ((xi,) * 3, "fp64", "direct"), (MESHES["uniform11x9x7"](), "fp32", "direct")]
    for mesh, precision, kernel in cases:
        s = pkg.Solver(*mesh, Ra=1e6, precision=precision)
        assert s.info.kernel == pkg.KERNELS[kernel], (precision, kernel)
        s.close()
    # too few nodes across for the staged window: the direct kernel
    small = O.mesh_tanh(5, 1.5)
    s = pkg.Solver(small, small, small, Ra=1e6, precision="fp32", kernel="tma3d")
    assert s.info.kernel == pkg.KERNELS["direct"]
    s.close()
    # the 3-D kernel on a 2-D mesh is an argument error
    with pytest.raises(pkg.IslbmError):
        pkg.Solver(xi, xi, Ra=1e6, precision="fp32", kernel="tma3d")


def test_full_size_256_cube_pipelined_equals_direct_and_conserves_mass():
    """The 3-D workload at its full size (256^3 tanh mesh, FP32, the bench's
    launch configuration): from smooth random T, u, v, w (equilibrium
    initialisation) three steps of the pipelined kernel agree with the direct
    kernel (checked against the oracle on smaller meshes above) on every node,
    and conserve mass to FP32 rounding.  The FP64 oracle needs ~20 s and
    ~15 GB per step at this size, so the comparison is kernel against kernel
    plus the invariant."""
    from synthetic import smooth_field
    n = 256
    xi = O.mesh_tanh(n, 1.5)
    shape = (n, n, n)
    T = smooth_field(shape, seed=41, amplitude=0.4, modes=2)
    vel = [smooth_field(shape, seed=42 + k, amplitude=0.01, modes=2) for k in range(3)]
    out = {}
    for kernel in ("tma3d", "direct"):
        s = pkg.Solver(xi, xi, xi, Ra=1e7, precision="fp32", kernel=kernel)
        s.set_fields(T, *vel)
        m0 = s.reduce()["mass"]
        s.step(3)
        out[kernel] = (s.fields(), m0, s.reduce()["mass"])
        s.close()
    fa, m0, m3 = out["tma3d"]
    fb, _, _ = out["direct"]
    assert rel_field_error(fa["T"], fb["T"]) <= 1e-6
    assert rel_vector_error([fa[k] for k in "uvw"], [fb[k] for k in "uvw"]) <= 1e-6
    assert abs(m3 - m0) <= 1e-6 * abs(m0)

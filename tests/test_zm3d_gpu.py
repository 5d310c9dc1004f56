"""The z-marching 3-D step kernels (zm3d: 32 x 8 columns, zm3d_t4: 32 x 4).

They apply the direct kernel's operations in the same order, so on the same
state they must give the direct kernel's populations; against the FP64 oracle
they are held to the tolerances of the other 3-D kernels (1e-5 field-relative
in FP32; 5e-6 / 5e-3 / 5e-2 of the largest population for far-from-equilibrium
states in FP32 / FP16 / BF16 storage).  Meshes span several columns in x and y,
ragged last columns and rows, and z chunks of several lengths.
"""
import os

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

ZM = ["zm3d", "zm3d_t4"]
POP_TOL = {"fp32": 5e-6, "fp16dev": 5e-3, "bf16dev": 5e-2}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cavity3d_tanh64.npz")


def _same_unit(ref, xi):
    """xi rescaled to the lattice unit (first spacing) of ref: every axis of a
    cavity uses one lattice unit."""
    return xi * ((ref[1] - ref[0]) / (xi[1] - xi[0]))


def meshes(name):
    if name == "erf36":
        return (O.mesh_erf(36, 1.5),) * 3
    if name == "ragged41x19x13":
        x = O.mesh_tanh(41, 1.5)
        return x, _same_unit(x, O.mesh_erf(19, 1.5)), _same_unit(x, O.mesh_tanh(13, 1.5))
    if name == "thin70x9x5":
        x = O.mesh_tanh(70, 1.5)
        return x, _same_unit(x, O.mesh_tanh(9, 1.5)), _same_unit(x, O.mesh_tanh(5, 1.5))
    raise KeyError(name)


@pytest.mark.parametrize("kernel", ZM)
@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("mesh", ["erf36", "ragged41x19x13"])
def test_random_state_against_oracle(mesh, precision, kernel):
    xi = meshes(mesh)
    cav = O.Cavity(*xi, params=O.Params(Ra=1e6))
    f = random_populations(19, cav.shape, seed=51, spread=0.2)
    g = random_signed(7, cav.shape, seed=52, amplitude=0.08)
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


def _populations(xi, precision, kernel, steps, seed=61):
    shape = tuple(len(x) - 2 for x in reversed(xi))
    f = random_populations(19, shape, seed=seed, spread=0.2)
    g = random_signed(7, shape, seed=seed + 1, amplitude=0.08)
    s = pkg.Solver(*xi, Ra=1e7, precision=precision, kernel=kernel)
    s.set_populations(f, g)
    s.step(steps)
    out = s.populations()
    s.close()
    return out


# FP32: the operations of the direct kernel in the same order (the compiler may
# still contract a product into a sum differently in the two kernels); 16-bit
# storage: one such FP32 difference can flip a stochastic rounding decision,
# one storage ulp, which the next steps carry along
SAME_TOL = {"fp32": 1e-6, "bf16dev": 5e-2}


@pytest.mark.parametrize("kernel", ZM)
@pytest.mark.parametrize("precision", ["fp32", "bf16dev"])
@pytest.mark.parametrize("mesh", ["erf36", "ragged41x19x13", "thin70x9x5"])
def test_same_populations_as_the_direct_kernel(mesh, precision, kernel):
    """After 20 steps from a random state the populations agree with the direct
    kernel's (the kernel checked against the oracle elsewhere)."""
    xi = meshes(mesh)
    fa, ga = _populations(xi, precision, kernel, 20)
    fb, gb = _populations(xi, precision, "direct", 20)
    scale = max(np.abs(fb).max(), np.abs(gb).max())
    assert np.abs(fa - fb).max() <= SAME_TOL[precision] * scale
    assert np.abs(ga - gb).max() <= SAME_TOL[precision] * scale


def test_cavity_64_against_the_stored_oracle_run():
    """64^3 tanh cavity, Ra = 1e6, 1000 steps from the seeded rest state: two
    columns in x, eight (zm3d) or sixteen (zm3d_t4) in y and several z chunks.
    The oracle's fields at 6000 sampled nodes and its reductions are stored
    (tests/golden/make_cavity3d_tanh64.py)."""
    ref = np.load(GOLDEN)
    n, steps = int(ref["n"]), int(ref["steps"])
    xi = O.mesh_tanh(n, float(ref["a"]))
    idx = ref["index"]
    red_ref = dict(zip([str(k) for k in ref["red_keys"]], ref["red_values"]))
    for kernel in ZM + ["tma3d"]:
        s = pkg.Solver(xi, xi, xi, Ra=float(ref["Ra"]), precision="fp32", kernel=kernel)
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
        s.step(steps)
        got = s.fields()
        red = s.reduce()
        s.close()
        eT = np.abs(got["T"].ravel()[idx] - ref["T"]).max() / float(ref["T_absmax"])
        eu = max(np.abs(got[k].ravel()[idx] - ref[k]).max() for k in "uvw") / float(ref["speed_max"])
        assert eT <= 1e-5 and eu <= 1e-5, (kernel, eT, eu)
        for k in ("Nu", "Nu_hot", "Nu_cold", "Re"):
            assert abs(red[k] - red_ref[k]) <= 1e-4 * max(1.0, abs(red_ref[k])), (kernel, k)


def test_full_size_256_cube_equals_direct_and_conserves_mass():
    """The 3-D workload at its full size (256^3 tanh mesh, FP32, the bench's
    launch configuration) from smooth random fields: three steps of the
    z-marching kernel agree with the direct kernel on every node and conserve
    mass to FP32 rounding (the FP64 oracle needs ~15 GB and ~20 s per step
    here; it checks both kernels on the smaller meshes above)."""
    from synthetic import smooth_field
    n = 256
    xi = O.mesh_tanh(n, 1.5)
    shape = (n, n, n)
    T = smooth_field(shape, seed=41, amplitude=0.4, modes=2)
    vel = [smooth_field(shape, seed=42 + k, amplitude=0.01, modes=2) for k in range(3)]
    out = {}
    for kernel in ("zm3d", "direct"):
        s = pkg.Solver(xi, xi, xi, Ra=1e7, precision="fp32", kernel=kernel)
        s.set_fields(T, *vel)
        m0 = s.reduce()["mass"]
        s.step(3)
        out[kernel] = (s.fields(), m0, s.reduce()["mass"])
        s.close()
    fa, m0, m3 = out["zm3d"]
    fb, _, _ = out["direct"]
    assert rel_field_error(fa["T"], fb["T"]) <= 1e-6
    assert rel_vector_error([fa[k] for k in "uvw"], [fb[k] for k in "uvw"]) <= 1e-6
    assert abs(m3 - m0) <= 1e-6 * abs(m0)

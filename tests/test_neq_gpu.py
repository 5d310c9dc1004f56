"""Non-equilibrium 16-bit storage (ISLBM_FP16NEQ) against the FP64 oracle.

Per node the state holds its moments (drho, jx, jy, T) in FP32 and, per
population, the remainder beyond the equilibrium of those moments in FP16
(scaled by 2^12, rounded to nearest).  Far from equilibrium (random
populations) the remainder is as large as the deviation itself, so one store
errs by up to 2^-11 of it, as FP16 deviations do: the population tolerance is
FP16DEV's 5e-3.  Near equilibrium (the cavity) the remainder is orders of
magnitude below the deviation: the bound used here is derived in
`_cavity_bound` from the oracle's own state.
"""
import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import temperature_noise
from tests.helpers import gpu_available, rel_field_error, rel_vector_error
from tests.test_parity_2d import MESHES, _random_state, oracle_run

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

POP_TOL = 5e-3


@pytest.mark.parametrize("kernel", ["tma_r2s2", "tma_r2s3"])
@pytest.mark.parametrize("mesh", ["erf45", "uniform37x29", "tanh64"])
@pytest.mark.parametrize("steps", [0, 1, 3])
def test_random_state_populations(mesh, kernel, steps):
    """Every population after 0 (encode and decode only), 1 and 3 steps from a
    far-from-equilibrium random state, ragged and tile-aligned meshes."""
    xi_x, xi_y = MESHES[mesh]()
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=1e6))
    f, g = _random_state(9, 5, cav.shape, seed=11)
    cav.init_populations(f, g)
    cav.step(steps)
    fp_ref, gp_ref = cav.post_collision()
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision="fp16neq", kernel=kernel)
    assert s.info.kernel == pkg.KERNELS[kernel]
    s.set_populations(f, g)
    s.step(steps)
    fp, gp = s.populations()
    s.close()
    assert np.abs(fp - fp_ref).max() / np.abs(fp_ref).max() <= POP_TOL
    assert np.abs(gp - gp_ref).max() / np.abs(gp_ref).max() <= POP_TOL


def test_other_kernels_and_3d_are_refused():
    xi = O.mesh_tanh(32, 1.5)
    for k in ("direct", "tiled", "tma_r4s2", "tma_r4s3"):
        with pytest.raises(pkg.IslbmError) as e:
            pkg.Solver(xi, xi, Ra=1e6, precision="fp16neq", kernel=k)
        assert e.value.status == 1
    with pytest.raises(pkg.IslbmError) as e:
        pkg.Solver(xi, xi, xi, Ra=1e5, precision="fp16neq")
    assert e.value.status == 1
    s = pkg.Solver(xi, xi, Ra=1e6, precision="fp16neq")
    with pytest.raises(pkg.IslbmError):
        s.set_row_range(0, 16)
    s.close()


def _remainder_ratios(f, g, a_T):
    """(max|r| / max|d|) of the flow and of the temperature populations of an
    oracle post-collision state: d_i the deviations, r_i = d_i - E_i(m) the
    part beyond the equilibrium of the node's moments, with rho = 1 in its
    quadratic terms (what FP16NEQ keeps in 16 bits)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])[:, None, None]
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])[:, None, None]
    d = f - w
    drho = d.sum(0)
    jx, jy = (ex * d).sum(0), (ey * d).sum(0)
    ej = ex * jx + ey * jy
    E = w * (drho + 3 * ej + 4.5 * ej ** 2 - 1.5 * (jx ** 2 + jy ** 2))
    T = g.sum(0)
    t0, ti = (1 - a_T) / 5, (4 + a_T) / 20
    cx = np.array([0, 1, 0, -1, 0])[:, None, None]
    cy = np.array([0, 0, 1, 0, -1])[:, None, None]
    Eg = np.where(np.arange(5)[:, None, None] == 0, t0, ti) * T + 0.5 * (cx * jx + cy * jy) * T
    return np.abs(d - E).max() / np.abs(d).max(), np.abs(g - Eg).max() / np.abs(g).max()


def _cavity_bound(steps):
    """Field tolerance after `steps` steps of the 64^2 Ra = 1e6 cavity.  One
    store errs by at most 2^-12 max|r| (FP16 round to nearest of r * 2^12,
    unit roundoff 2^-11), against 2^-24 max|d| for an FP32 store; the FP32
    path meets 1e-5 after 1000 steps, so the bound is 1e-5 times the larger
    of the two lattices' ratios 2^12 max|r| / max|d| (at least 1: the FP32
    moments round as FP32 stores do)."""
    xi = O.mesh_tanh(64, 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=1e6))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(steps)
    f, g = cav.post_collision()
    rf, rg = _remainder_ratios(f, g, cav.par.a_T)
    return 1e-5 * max(1.0, 2.0 ** 12 * max(rf, rg)), rf, rg


def test_cavity_1000_steps_against_the_oracle():
    tol, rf, rg = _cavity_bound(1000)
    ref = oracle_run("tanh64", 1e6, 1000)
    xi_x, xi_y = MESHES["tanh64"]()
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision="fp16neq")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(1000)
    got = s.fields()
    red = s.reduce()
    s.close()
    eT = rel_field_error(got["T"], ref["T"])
    eu = rel_vector_error([got["u"], got["v"]], [ref["u"], ref["v"]])
    eNu = abs(red["Nu"] / ref["red"]["Nu"] - 1)
    print(f"fp16neq 1000 steps: |r|/|d| flow {rf:.2e} temperature {rg:.2e}, bound {tol:.2e}: "
          f"T {eT:.3e} u {eu:.3e} Nu {eNu:.3e}")
    assert eT <= tol and eu <= tol and eNu <= tol


def test_batch_members_equal_single_solvers_bitwise():
    """A batch of FP16NEQ cavities (one persistent launch) against the same
    cavities stepped alone with the same kernel: identical bits."""
    cavs = [dict(n=48, mesh="tanh", Ra=1e6), dict(n=64, mesh="erf", Ra=3e6),
            dict(n=45, mesh="uniform", Ra=1e5)]
    b = pkg.Batch(cavs, precision="fp16neq", autotune=True)
    for k, m in enumerate(b.members):
        assert b.tile_rows(k) == 8
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    b.step(64 + 64 + 9)
    b.synchronize()
    for k, (c, m) in enumerate(zip(cavs, b.members)):
        xi = (pkg.islbm_mesh_uniform(c["n"]) if c["mesh"] == "uniform"
              else getattr(pkg, "islbm_mesh_" + c["mesh"])(c["n"], 1.5))
        s = pkg.Solver(xi, xi, Ra=c["Ra"], precision="fp16neq", kernel="tma_r2s2")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=k))
        s.step(137)
        fa, ga = m.populations()
        fb, gb = s.populations()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ga, gb)
        s.close()
    b.close()

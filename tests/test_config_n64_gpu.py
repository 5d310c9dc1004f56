"""The small parity workload end to end: 2-D cavity, Ra = 1e6, 64^2 tanh mesh
(a = 1.5), rest with the seeded 1e-6 noise on T, 20,000 steps, every storage
precision against the FP64 oracle.

Bounds.  FP64: both sides round at 1e-16 per operation in different orders;
over 20,000 steps of a steady, non-chaotic flow the difference grows roughly
linearly in the number of steps from the 1e-12-level seen after 1000 steps,
so 1e-9 field-relative.  FP32: 1e-5 after 1000 steps grows to at most ~1e-4.
FP16 / BF16 deviations (stochastically rounded, unit roundoff 2^-11 / 2^-8 of
values ~1e-2): the fields are checked at 2e-2 / 1e-1 and Nu at 2% / 5%; the
measured errors are printed for the record.  FP16NEQ (FP32 moments, FP16
remainders at least ten times smaller than the deviations) is held to the
FP16 bounds.
"""
import functools

import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import temperature_noise
from tests.helpers import gpu_available, rel_field_error, rel_vector_error

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

N, STEPS, RA = 64, 20_000, 1e6
FIELD_TOL = {"fp64": 1e-9, "fp32": 1e-4, "fp16dev": 2e-2, "bf16dev": 1e-1, "fp16neq": 2e-2}
NU_TOL = {"fp64": 1e-9, "fp32": 1e-4, "fp16dev": 2e-2, "bf16dev": 5e-2, "fp16neq": 2e-2}


@functools.lru_cache(maxsize=None)
def oracle_state():
    x = O.mesh_tanh(N, 1.5)
    cav = O.Cavity(x, x, params=O.Params(Ra=RA))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(STEPS)
    rho, u, T = cav.fields()
    return T, u, cav.reductions()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev", "bf16dev", "fp16neq"])
def test_n64_workload_against_oracle(precision):
    T, u, red_ref = oracle_state()
    xi = pkg.islbm_mesh_tanh(N, 1.5)
    s = pkg.Solver(xi, xi, Ra=RA, precision=precision)
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(STEPS)
    got = s.fields()
    red = s.reduce()
    s.close()
    eT = rel_field_error(got["T"], T)
    eu = rel_vector_error([got["u"], got["v"]], [u[0], u[1]])
    eNu = abs(red["Nu"] / red_ref["Nu"] - 1)
    eRe = abs(red["Re"] / red_ref["Re"] - 1)
    print(f"{precision}: T {eT:.3e}  u {eu:.3e}  Nu {eNu:.3e}  Re {eRe:.3e}")
    assert eT <= FIELD_TOL[precision] and eu <= FIELD_TOL[precision], (eT, eu)
    assert eNu <= NU_TOL[precision] and eRe <= NU_TOL[precision], (eNu, eRe)

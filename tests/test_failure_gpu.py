"""Failure detection on the GPU without a fault: the bounded waits of the
pipelined kernels give up on a barrier that never completes, report
ISLBM_ERR_TIMEOUT through the device flag, and leave the context usable."""
import time

import numpy as np
import pytest

from oracle import islbm_oracle as O
from synthetic import temperature_noise
from tests.helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA device")]


def test_bounded_wait_times_out_and_the_context_survives():
    import paper_2509_01099_gb300 as pkg
    t0 = time.perf_counter()
    st = pkg.islbm_selftest_wait_timeout()
    elapsed = time.perf_counter() - t0
    assert st == 6, st                       # ISLBM_ERR_TIMEOUT
    assert elapsed < 5.0, elapsed            # the wait limit is one second
    # the same process keeps computing correctly afterwards
    xi = O.mesh_tanh(24, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e5, precision="fp32")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(100)
    r = s.reduce()
    s.close()
    assert r["status"] == 0 and np.isfinite(r["Nu"])


def test_abort_flag_ends_the_other_warps_waits():
    """The CTA abort flag of the barrier-free pipelined loops: after warp 0's
    wait gives up and raises the flag, the other warps' three waits on an
    mbarrier that never completes take about one wait limit in all (the
    second and third end at once), not three."""
    import paper_2509_01099_gb300 as pkg
    t0 = time.perf_counter()
    st, failed, ms = pkg.islbm_selftest_wait_abort()
    elapsed = time.perf_counter() - t0
    assert st == 6, st                       # ISLBM_ERR_TIMEOUT from warp 0
    assert failed == 3, failed
    assert 900 <= ms < 2000, ms              # one limit of 1 s, not three
    assert elapsed < 5.0, elapsed
    xi = O.mesh_tanh(24, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e5, precision="fp32")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    s.step(100)
    r = s.reduce()
    s.close()
    assert r["status"] == 0 and np.isfinite(r["Nu"])

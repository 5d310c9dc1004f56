"""The allocation-free reduction entry point, islbm_reduce_noalloc.

Some callers of this library cannot allocate device memory: their memory pool
is fully reserved, or they run where an allocation (and the device
synchronisation it can cause) is not allowed.  islbm_reduce_noalloc serves
them: it takes the state and the meshes in the caller's own device memory and
keeps its scratch in a fixed static device array.  These tests call it through
the C ABI and check it against islbm_reduce, the entry point that uses the
handle's scratch, with the tolerance of the FP64 parity tests (1e-10
relative), on two calls in a row.  The file is named to run last.
"""
import numpy as np
import pytest

from synthetic import temperature_noise
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

KEYS = ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re", "mass", "ke", "max_speed")


def _close(a, b, tol=1e-10):
    return abs(a - b) <= tol * max(abs(b), 1e-30)


@pytest.mark.parametrize("n, mesh, steps", [(64, "tanh", 400), (45, "erf", 250)])
def test_noalloc_reduction_matches_islbm_reduce_twice(n, mesh, steps):
    import torch
    xi = getattr(pkg, "islbm_mesh_" + mesh)(n, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e6, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=2))
    s.step(steps)
    ref = s.reduce()
    f, g = s.populations()                      # full FP64 post-collision state
    s.close()
    df = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    dg = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    dxi = torch.from_numpy(xi).cuda()
    for call in range(2):                        # the second call reuses the scratch
        got = pkg.islbm_reduce_noalloc(df, dg, n, n, dxi, dxi, 1e6, 0.71)
        for k in KEYS:
            assert _close(got[k], ref[k]), (call, k, got[k], ref[k])
        assert got["nonfinite"] == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.IslbmError) as e:
        pkg.islbm_reduce_noalloc(t, t, 20000, 20000, t, t, 1e6, 0.71)
    assert e.value.status == 1
    assert "134217728" in str(e.value)

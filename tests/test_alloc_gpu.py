"""Where the library's device memory comes from (islbm_set_allocator).

Every device allocation of a handle, a batch and the network GEMM's split-K
workspace goes through the registered allocator (the binding registers
torch's caching allocator), or cudaMallocAsync on the owner's stream when none
is registered.  A counting allocator checks that every allocation is made
through it and returned; the results do not depend on the allocator.
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


class Counting:
    def __init__(self):
        self.alloc, self.release = pkg.torch_allocator()
        self.live, self.n_alloc, self.n_free = {}, 0, 0

    def a(self, nbytes, device, stream):
        p = self.alloc(nbytes, device, stream)
        self.live[p] = nbytes
        self.n_alloc += 1
        return p

    def r(self, ptr, device, stream):
        assert ptr in self.live, "freed a pointer it did not allocate"
        del self.live[ptr]
        self.n_free += 1
        self.release(ptr, device, stream)


def _run(n=96):
    xi = pkg.islbm_mesh_tanh(n, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e7, precision="fp32")
    s.set_fields(temperature_noise(s.shape, 1e-4, seed=8))
    s.step(70)                     # a 64-step graph and 6 launches
    f = s.fields()
    red = s.reduce()
    s.steady_change()              # allocates the snapshot
    s.average_reset()              # and the time-average accumulators
    s.close()
    return f, red


def test_handles_and_batches_use_the_registered_allocator():
    c = Counting()
    pkg.islbm_set_allocator(c.a, c.r)
    try:
        f1, r1 = _run()
        assert c.n_alloc >= 8 and not c.live and c.n_free == c.n_alloc
        b = pkg.Batch([dict(n=64, mesh="tanh", Ra=1e6), dict(n=80, mesh="tanh", Ra=1e7)], "fp32")
        b.step(10)
        b.synchronize()
        assert c.live
        b.close()
        assert not c.live
    finally:
        pkg.islbm_set_allocator(*pkg.torch_allocator())
    # the default path: cudaMallocAsync / cudaFreeAsync on the handle's stream
    pkg.islbm_set_allocator(None, None)
    try:
        f2, r2 = _run()
    finally:
        pkg.islbm_set_allocator(*pkg.torch_allocator())
    for k in f1:
        np.testing.assert_array_equal(f1[k], f2[k])
    assert r1["Nu"] == r2["Nu"]


def test_a_failed_allocation_is_reported_as_out_of_memory():
    pkg.islbm_set_allocator(lambda n, d, s: 0, lambda p, d, s: None)
    try:
        xi = pkg.islbm_mesh_tanh(32, 1.5)
        with pytest.raises(pkg.IslbmError) as e:
            pkg.Solver(xi, xi, Ra=1e6, precision="fp32")
        assert e.value.status == 3          # ISLBM_ERR_OOM
    finally:
        pkg.islbm_set_allocator(*pkg.torch_allocator())



class NanFilled:
    """Hands out blocks filled with 0xFF bytes (NaN in every float format), as a
    pooled allocator may return a block that held anything before."""

    def __init__(self):
        self.live = {}

    def a(self, nbytes, device, stream):
        import torch
        t = torch.full((max(int(nbytes), 1),), 255, dtype=torch.uint8, device=f"cuda:{device}")
        torch.cuda.synchronize(device)
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def r(self, ptr, device, stream):
        import torch
        torch.cuda.synchronize(device)
        del self.live[ptr]


@pytest.mark.parametrize("dim", [2, 3])
def test_recycled_memory_never_reaches_the_state(dim):
    """Every buffer the library allocates is zeroed or written before it is
    read: with all allocations filled with NaN, the first steady-state check,
    the steps and the reductions stay finite and equal those on fresh memory."""
    def run():
        if dim == 2:
            xi = pkg.islbm_mesh_tanh(48, 1.5)
            s = pkg.Solver(xi, xi, Ra=1e6, precision="fp32")
        else:
            xi = pkg.islbm_mesh_tanh(24, 1.5)
            s = pkg.Solver(xi, xi, xi, Ra=1e5, precision="fp32")
        s.set_fields(temperature_noise(s.shape, 1e-4, seed=5))
        first = s.steady_change()        # no snapshot yet: must not read the buffer
        s.step(40)
        second = s.steady_change()
        red = s.reduce()
        f = s.fields()
        s.close()
        return first, second, red, f

    nan = NanFilled()
    pkg.islbm_set_allocator(nan.a, nan.r)
    try:
        a1, b1, r1, f1 = run()
    finally:
        pkg.islbm_set_allocator(*pkg.torch_allocator())
    assert not nan.live
    a2, b2, r2, f2 = run()
    assert tuple(a1) == tuple(a2) and tuple(b1) == tuple(b2)
    assert np.isfinite(b1).all() and np.isfinite(r1["Nu"]) and r1["Nu"] == r2["Nu"]
    for k in f1:
        np.testing.assert_array_equal(f1[k], f2[k])

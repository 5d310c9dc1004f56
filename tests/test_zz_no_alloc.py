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


def _close(a, b, tol=1e-10, floor=1e-30):
    return abs(a - b) <= tol * max(abs(b), floor)


def _meshes(nx, ny, mesh):
    """x and y meshes of one lattice unit (the y mesh rescaled to x's first spacing)."""
    mk = getattr(pkg, "islbm_mesh_" + mesh)
    xi_x, xi_y = mk(nx, 1.5), mk(ny, 1.5)
    return xi_x, xi_y * ((xi_x[1] - xi_x[0]) / (xi_y[1] - xi_y[0]))


# One block reduces 16,384 nodes: 64^2 and 45^2 are one block, 256^2 four full
# blocks, 130 x 260 three blocks with a partial last one (the fixed-order sum
# of several partial rows).
@pytest.mark.parametrize("nx, ny, mesh, steps",
                         [(64, 64, "tanh", 400), (45, 45, "erf", 250), (256, 256, "tanh", 200),
                          (130, 260, "erf", 200)])
def test_noalloc_reduction_matches_islbm_reduce_twice(nx, ny, mesh, steps):
    import torch
    xi_x, xi_y = _meshes(nx, ny, mesh)
    s = pkg.Solver(xi_x, xi_y, Ra=1e6, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=2))
    s.step(steps)
    ref = s.reduce()
    f, g = s.populations()                      # full FP64 post-collision state
    s.close()
    df = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    dg = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    dxx, dxy = torch.from_numpy(xi_x).cuda(), torch.from_numpy(xi_y).cuda()
    for call in range(2):                        # the second call reuses the scratch
        got = pkg.islbm_reduce_noalloc(df, dg, nx, ny, dxx, dxy, 1e6, 0.71)
        for k in KEYS:
            # Nusselt numbers are O(1) quantities: early in a run Nu_middle can
            # sit near zero, where its rounding is relative to 1, not to itself
            floor = 1.0 if k.startswith("Nu") else 1e-30
            assert _close(got[k], ref[k], floor=floor), (call, k, got[k], ref[k])
        assert got["nonfinite"] == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    a = t.data_ptr()      # raw addresses: the binding's size checks do not apply
    with pytest.raises(pkg.IslbmError) as e:
        pkg.islbm_reduce_noalloc(a, a, 20000, 20000, a, a, 1e6, 0.71)
    assert e.value.status == 1
    assert "134217728" in str(e.value)


def test_noalloc_rejects_meshes_with_different_lattice_units():
    """islbm_create refuses such meshes; the allocation-free reduction finds the
    mismatch on the device and returns ISLBM_ERR_ARG instead of a result."""
    import torch
    n = 32
    xi = pkg.islbm_mesh_tanh(n, 1.5)
    s = pkg.Solver(xi, xi, Ra=1e6, precision="fp64")
    s.set_fields(temperature_noise(s.shape, 1e-6, seed=2))
    s.step(10)
    f, g = s.populations()
    s.close()
    df = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    dg = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    dx = torch.from_numpy(xi).cuda()
    dy = torch.from_numpy(xi * 1.5).cuda()       # same shape, larger lattice unit
    with pytest.raises(pkg.IslbmError) as e:
        pkg.islbm_reduce_noalloc(df, dg, n, n, dx, dy, 1e6, 0.71)
    assert e.value.status == 1 and "lattice unit" in str(e.value)
    # a correct call right after still gives the handle's result
    got = pkg.islbm_reduce_noalloc(df, dg, n, n, dx, dx, 1e6, 0.71)
    assert got["nonfinite"] == 0

"""The slab calls of the library on one GPU (islbm_set_row_range,
islbm_get_rows / islbm_set_rows, islbm_reduce_sums / islbm_finish_sums).

Two and three slabs of one cavity, one handle each, share the GPU and
exchange their halo rows through device buffers between steps
(paper_2509_01099_gb300.decomp.step_in_process); no kernel waits on another.
Each slab's rows must equal an undivided handle's bit for bit after the run,
for the TMA kernels and the direct kernel, in FP32 and 16-bit storage; the
combined partial sums must finish to the undivided reductions.
"""
import numpy as np
import pytest

from paper_2509_01099_gb300 import decomp as D
from synthetic import temperature_noise
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

if gpu_available():
    from paper_2509_01099_gb300 import build as _B
    _B.build()
import paper_2509_01099_gb300 as pkg  # noqa: E402

NX, NY, STEPS = 150, 137, 70


def _solver(precision, kernel):
    xi_x = pkg.islbm_mesh_tanh(NX, 1.5)
    xi_y = pkg.islbm_mesh_tanh(NY, 1.5)
    xi_y = xi_y * ((xi_x[1] - xi_x[0]) / (xi_y[1] - xi_y[0]))
    s = pkg.Solver(xi_x, xi_y, Ra=1e8, precision=precision, kernel=kernel)
    s.set_fields(temperature_noise(s.shape, 1e-3, seed=5))
    s.step(40)                      # a developed, non-trivial state
    return s


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision,kernel", [("fp32", "tma_r2s2"), ("fp32", "tma_r4s3"),
                                              ("fp32", "direct"), ("fp64", "direct"),
                                              ("bf16dev", "tma_r4s2"), ("fp32", "tiled")])
def test_slabs_on_one_gpu_equal_the_undivided_handle(world, precision, kernel):
    import torch
    ref = _solver(precision, kernel)
    slabs = [_solver(precision, kernel) for _ in range(world)]
    plan = D.SlabPlan(NY, world)
    for r, s in enumerate(slabs):
        s.set_row_range(*plan.rows(r))
    bufs = D.make_buffers(slabs, plan,
                          lambda nb: torch.empty(nb, dtype=torch.uint8, device="cuda"))
    D.step_in_process(slabs, plan, STEPS, bufs)
    ref.step(STEPS)
    f_ref, g_ref = ref.populations()
    sums = []
    for r, s in enumerate(slabs):
        r0, r1 = plan.rows(r)
        f, g = s.populations()
        np.testing.assert_array_equal(f[:, r0:r1], f_ref[:, r0:r1])
        np.testing.assert_array_equal(g[:, r0:r1], g_ref[:, r0:r1])
        sums.append(s.reduce_sums())
    # the reductions: combined slab sums against the undivided handle
    red = slabs[0].finish_sums(D.combine_sums(sums))
    want = ref.reduce()
    for k in ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re", "mass", "max_speed"):
        assert abs(red[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), (k, red[k], want[k])
    with pytest.raises(pkg.IslbmError):
        slabs[0].reduce()               # a slab's own reduce would be partial
    for s in slabs + [ref]:
        s.close()


def test_row_range_arguments():
    s = _solver("fp32", "auto")
    for r0, r1 in ((-1, 5), (5, 5), (0, NY + 1), (9, 3)):
        with pytest.raises(pkg.IslbmError):
            s.set_row_range(r0, r1)
    s.set_row_range(0, NY)                # the whole range: an undivided handle again
    s.reduce()
    with pytest.raises(ValueError):
        s.get_rows(0, 2, np.zeros(10, dtype=np.uint8))     # too small for two rows
    s.close()

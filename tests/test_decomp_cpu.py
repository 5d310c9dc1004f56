"""The slab decomposition's host logic on the CPU (paper_2509_01099_gb300.decomp).

The row split and the halo plan are checked directly.  The exchange runs on
two and three gloo ranks on 127.0.0.1 with the FP64 oracle as each rank's
step engine: every rank holds the whole mesh, but before each step it
poisons (NaN) every row but its slab and the two halo rows it has just
received, so its slab is right only if the exchange delivered the right rows.
After the run the slabs must equal the undivided oracle run bit for bit, and
the combined partial sums the undivided sums.
"""
import os
import socket

import numpy as np
import pytest

from oracle import islbm_oracle as O
from paper_2509_01099_gb300 import decomp as D
from synthetic import temperature_noise

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, STEPS = 14, 17, 25


def test_slab_plan_is_balanced_and_the_halo_plan_is_consistent():
    for ny, world in ((17, 2), (17, 3), (100, 7), (5, 5)):
        plan = D.SlabPlan(ny, world)
        sizes = [plan.rows(r)[1] - plan.rows(r)[0] for r in range(world)]
        assert sum(sizes) == ny and max(sizes) - min(sizes) <= 1
        assert plan.rows(0)[0] == 0 and plan.rows(world - 1)[1] == ny
        sent = {}
        for r in range(world):
            send, recv = plan.halo_plan(r)
            r0, r1 = plan.rows(r)
            for peer, row in send:
                assert r0 <= row < r1
                sent[(r, peer)] = row
            for peer, row in recv:
                assert row in (r0 - 1, r1)
        for r in range(world):
            for peer, row in plan.halo_plan(r)[1]:
                assert sent[(peer, r)] == row      # what the peer sends is what r expects
    with pytest.raises(ValueError):
        D.SlabPlan(3, 4)


def test_combine_sums_adds_all_but_the_maximum():
    a, b = np.arange(16.0), 10 * np.arange(16.0)
    b[13] = 1.0
    c = D.combine_sums([a, b])
    assert c[0] == 0 and c[5] == 55.0 and c[13] == 13.0


class OracleSlab:
    """Step engine of one rank in these tests: the oracle on the whole mesh,
    with every row outside the slab and its halo poisoned before each step."""

    def __init__(self, cav):
        self.cav = cav
        self.r0, self.r1 = 0, cav.shape[0]

    def set_row_range(self, r0, r1):
        self.r0, self.r1 = r0, r1

    def rows_bytes(self, nrows):
        return (self.cav.flow.q + self.cav.thermal.q) * nrows * self.cav.shape[1] * 8

    def synchronize(self):
        pass

    def get_rows(self, row, nrows, buf):
        v = np.concatenate([self.cav.f[:, row:row + nrows], self.cav.g[:, row:row + nrows]])
        buf.numpy().view(np.float64)[:] = v.ravel()

    def set_rows(self, row, nrows, buf):
        v = buf.numpy().view(np.float64).reshape(-1, nrows, self.cav.shape[1])
        q = self.cav.flow.q
        self.cav.f[:, row:row + nrows] = v[:q]
        self.cav.g[:, row:row + nrows] = v[q:]

    def step(self, n=1):
        keep = np.zeros(self.cav.shape[0], bool)
        keep[max(self.r0 - 1, 0):self.r1 + 1] = True
        with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
            self.cav.f[:, ~keep] = np.nan
            self.cav.g[:, ~keep] = np.nan
            self.cav.step(n)

    def reduce_sums(self):
        rho, u, T = (a[self.r0:self.r1] for a in _fields(self.cav))
        s = np.zeros(16)
        s[0], s[1], s[2] = rho.sum(), T.sum(), (u * u).sum()
        s[13] = np.abs(u).max()
        return s

    def finish_sums(self, sums, check=True):
        return {"sums": np.asarray(sums)}


def _fields(cav):
    with np.errstate(invalid="ignore"):
        rho, u, T = cav.fields()
    return rho, u[0], T


def _cavity():
    xi_x = O.mesh_tanh(NX, 1.5)
    xi_y = O.mesh_erf(NY, 1.5)
    xi_y = xi_y * ((xi_x[1] - xi_x[0]) / (xi_y[1] - xi_y[0]))
    cav = O.Cavity(xi_x, xi_y, params=O.Params(Ra=1e6))
    cav.init_fields(temperature_noise(cav.shape, 1e-3, seed=4))
    return cav


def _rank_main(rank, world, port, out, skip_exchange):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    eng = OracleSlab(_cavity())
    slab = D.Slab(eng, D.SlabPlan(NY, world), rank, D.TorchComm("cpu"))
    if skip_exchange:
        slab.exchange = lambda: None
    slab.step(STEPS)
    red = slab.reduce()
    out.put((rank, slab.r0, slab.r1, eng.cav.f[:, slab.r0:slab.r1].copy(),
             eng.cav.g[:, slab.r0:slab.r1].copy(), red["sums"]))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, skip_exchange=False):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, skip_exchange))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    return sorted(got, key=lambda t: t[0])


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_slabs_equal_the_undivided_run_bit_for_bit(world):
    ref = _cavity()
    ref.step(STEPS)
    full = OracleSlab(ref)
    ref_sums = full.reduce_sums()
    for rank, r0, r1, f, g, sums in _run(world):
        np.testing.assert_array_equal(f, ref.f[:, r0:r1])
        np.testing.assert_array_equal(g, ref.g[:, r0:r1])
        np.testing.assert_allclose(sums, ref_sums, rtol=1e-13, atol=0)


def test_slabs_without_the_exchange_go_wrong():
    """The poisoned rows reach the slabs when no halo is exchanged."""
    got = _run(2, skip_exchange=True)
    assert any(np.isnan(f).any() for _, _, _, f, _, _ in got)

"""Slab domain decomposition of the 2-D cavity over ranks (one GPU each).

The time step of Sec. 2.2 reads, at a node, the post-collision populations of
its own row and of the rows next to it (the y stencil of the quadratic
interpolation; the bounce-back partner at a wall lies in the node's own row).
Rows are therefore split into contiguous slabs, one per rank; before every
step each rank sends its first and last rows to the neighbouring ranks and
receives the rows just outside its slab (one halo row per side).  Every rank
holds the whole mesh in its handle but steps only its slab
(islbm_set_row_range), so a slab's rows are computed from exactly the values a
single handle would use: the decomposed run gives the single-rank run's bits.
The reductions add the slabs' raw sums (one of them, the largest speed, by
max) and finish them once (islbm_reduce_sums / islbm_finish_sums).

Host logic only: the step and the row copies run in the library; the transport
is torch.distributed (NCCL between GPUs, gloo on the CPU) or, for slabs that
share a process, plain copies.
"""
from __future__ import annotations

import numpy as np

from .islbm import REDUCTION_SUMS, SUM_MAX_SLOT


class SlabPlan:
    """Contiguous, balanced row ranges [bounds[r], bounds[r+1]) of ny rows over
    `world` ranks."""

    def __init__(self, ny: int, world: int):
        if world < 1 or world > ny:
            raise ValueError(f"cannot split {ny} rows over {world} ranks")
        self.ny, self.world = int(ny), int(world)
        self.bounds = [(r * self.ny) // self.world for r in range(self.world + 1)]

    def rows(self, rank: int):
        return self.bounds[rank], self.bounds[rank + 1]

    def below(self, rank: int):
        return rank - 1 if rank > 0 else None

    def above(self, rank: int):
        return rank + 1 if rank < self.world - 1 else None

    def halo_plan(self, rank: int):
        """(send, recv) lists of (peer, row): the rows this rank sends to its
        neighbours (its first row down, its last row up) and the halo rows it
        receives (the row below its slab, the row above it)."""
        r0, r1 = self.rows(rank)
        send, recv = [], []
        if self.below(rank) is not None:
            send.append((self.below(rank), r0))
            recv.append((self.below(rank), r0 - 1))
        if self.above(rank) is not None:
            send.append((self.above(rank), r1 - 1))
            recv.append((self.above(rank), r1))
        return send, recv


def combine_sums(parts):
    """Reduction sums of disjoint slabs added up; the largest-speed entry by max."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    total = np.sum(parts, axis=0)
    total[SUM_MAX_SLOT] = max(p[SUM_MAX_SLOT] for p in parts)
    return total


class TorchComm:
    """Point-to-point and all-reduce over torch.distributed.  Buffers live on
    `device` (cuda for NCCL, cpu for gloo)."""

    def __init__(self, device="cpu", group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.device = torch.device(device)

    def buffer(self, nbytes: int):
        pin = self.device.type == "cpu" and self.torch.cuda.is_available()
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device,
                                pin_memory=pin)

    def exchange(self, sends, recvs):
        """sends / recvs: lists of (peer, tensor); all complete on return."""
        reqs = [self.dist.irecv(t, src=peer, group=self.group) for peer, t in recvs]
        reqs += [self.dist.isend(t, dst=peer, group=self.group) for peer, t in sends]
        for r in reqs:
            r.wait()

    def allreduce_sums(self, sums):
        t = self.torch.tensor(np.asarray(sums, dtype=np.float64))
        mx = t[SUM_MAX_SLOT].clone().reshape(1)
        t[SUM_MAX_SLOT] = 0.0
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        self.dist.all_reduce(mx, op=self.dist.ReduceOp.MAX, group=self.group)
        out = t.numpy().copy()
        out[SUM_MAX_SLOT] = float(mx.item())
        return out


class Slab:
    """One rank's part of a decomposed cavity.

    engine: a Solver (or an object with its slab methods: set_row_range,
    rows_bytes, get_rows, set_rows, synchronize, step, reduce_sums,
    finish_sums) holding the whole mesh; comm: a TorchComm."""

    def __init__(self, engine, plan: SlabPlan, rank: int, comm):
        self.engine, self.plan, self.rank, self.comm = engine, plan, int(rank), comm
        self.r0, self.r1 = plan.rows(rank)
        engine.set_row_range(self.r0, self.r1)
        self.send, self.recv = plan.halo_plan(rank)
        nb = engine.rows_bytes(1)
        self.sbuf = [(peer, comm.buffer(nb)) for peer, _ in self.send]
        self.rbuf = [(peer, comm.buffer(nb)) for peer, _ in self.recv]

    def exchange(self):
        """Refresh the halo rows of the current state from the neighbours."""
        for (peer, row), (_, buf) in zip(self.send, self.sbuf):
            self.engine.get_rows(row, 1, buf)
        self.engine.synchronize()
        self.comm.exchange(self.sbuf, self.rbuf)
        for (peer, row), (_, buf) in zip(self.recv, self.rbuf):
            self.engine.set_rows(row, 1, buf)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            self.engine.step(1)

    def reduce(self, check: bool = True) -> dict:
        """The finished reductions of the whole cavity (every rank gets them)."""
        total = self.comm.allreduce_sums(self.engine.reduce_sums())
        return self.engine.finish_sums(total, check)


def step_in_process(engines, plan: SlabPlan, n: int = 1, buffers=None):
    """Slabs that share one process (one handle per slab, e.g. on one GPU):
    each step copies every rank's boundary rows into its neighbours' halos
    through `buffers` (one per rank and side, from make_buffers), then steps
    every slab.  No kernel waits on another: the copies and the steps are
    ordered by the host."""
    for _ in range(int(n)):
        for rank, eng in enumerate(engines):
            send, _ = plan.halo_plan(rank)
            for peer, row in send:
                eng.get_rows(row, 1, buffers[(rank, peer)])
        for eng in engines:
            eng.synchronize()
        for rank, eng in enumerate(engines):
            _, recv = plan.halo_plan(rank)
            for peer, row in recv:
                eng.set_rows(row, 1, buffers[(peer, rank)])
        for eng in engines:
            eng.synchronize()
        for eng in engines:
            eng.step(1)


def make_buffers(engines, plan: SlabPlan, alloc):
    """One row buffer per (sender, receiver) pair; alloc(nbytes) makes one."""
    out = {}
    for rank, eng in enumerate(engines):
        send, _ = plan.halo_plan(rank)
        for peer, _row in send:
            out[(rank, peer)] = alloc(eng.rows_bytes(1))
    return out

"""Learned warm start of the 2-D side-heated cavity (not part of the paper).

The solver generates its own training data: a batch of cavities at training
Rayleigh numbers is stepped from rest and late-time snapshots of (T, u, v) are
packed into network channels on the device.  WarmStartNet is trained on them
with its own kernels (BF16 tensor-core GEMMs, FP32 accumulation, Adam), and
its prediction for a new Rayleigh number initialises a solver through the
equilibrium initialisation of Sec. 2.1 (islbm_set_fields_device), in place of
the rest state.  compare() runs the same held-out cavities from rest and from
the prediction to a steady Nu and reports the steps, the wall time and the
steady Nu / Re of both.

Everything that computes runs in the library's kernels; torch holds device
memory and gathers training minibatches (index_select).
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np

from .cnn import VEL_SCALE, WarmStartNet, features
from .islbm import Batch, IslbmError, islbm_set_fields_device, load_library

DEFAULT_N = 256
DEFAULT_A = 1.5


def _ck(st):
    if st != 0:
        raise IslbmError(st, "warm-start field conversion")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _scales(info):
    """(T_mid, T_scale, u_scale) of the channel encoding for a solver."""
    return 0.0, 1.0, info.u_f / VEL_SCALE


def cavities(ras, n=DEFAULT_N, a=DEFAULT_A, pr=0.71):
    return [{"n": n, "mesh": "tanh", "a": a, "Ra": float(r), "Pr": pr} for r in ras]


class _FieldBuffers:
    def __init__(self, nodes):
        import torch
        self.T = torch.empty(nodes, dtype=torch.float64, device="cuda")
        self.u = torch.empty_like(self.T)
        self.v = torch.empty_like(self.T)


def snapshot_dataset(ras, steps, snapshots=20, every=50_000, n=DEFAULT_N, a=DEFAULT_A, pr=0.71,
                     precision="fp32"):
    """Step a batch of cavities from rest and pack late-time snapshots.

    Snapshots of every cavity are taken at steps - (snapshots - 1 - j) * every,
    j = 0 .. snapshots-1.  Returns (data [len(ras) * snapshots, n, n, 3] FP32
    on the device, features [len(ras) * snapshots, 16], run log dict)."""
    import torch
    lib = load_library()
    first = steps - (snapshots - 1) * every
    if first <= 0:
        raise ValueError("steps must exceed (snapshots - 1) * every")
    batch = Batch(cavities(ras, n, a, pr), precision)
    nodes = n * n
    buf = _FieldBuffers(nodes)
    data = torch.empty((len(ras) * snapshots, n, n, 3), device="cuda")
    feats = np.repeat(features(np.log10(ras), [pr] * len(ras), [a] * len(ras)), snapshots, axis=0)
    log = {"first": first, "every": every, "steps": steps, "wall_s": 0.0, "du": []}
    t0 = time.perf_counter()
    batch.step(first)
    for j in range(snapshots):
        if j:
            batch.step(every)
        row = []
        for i, m in enumerate(batch.members):
            m.fields_device(T=buf.T, u=buf.u, v=buf.v)
            T_mid, T_scale, u_scale = _scales(m.info)
            dst = data[i * snapshots + j]
            _ck(lib.islbm_cnn_pack_fields(ctypes.c_void_p(buf.T.data_ptr()),
                                          ctypes.c_void_p(buf.u.data_ptr()),
                                          ctypes.c_void_p(buf.v.data_ptr()), nodes, T_mid,
                                          T_scale, u_scale, ctypes.c_void_p(dst.data_ptr()),
                                          _stream()))
            if j >= snapshots - 2:
                du = m.steady_change()[0]   # change between the last two snapshots
                if j == snapshots - 1:
                    row.append(du)
        if row:
            log["du"] = row
    batch.synchronize()
    torch.cuda.synchronize()
    log["wall_s"] = time.perf_counter() - t0
    batch.close()
    return data, feats, log


def train(net: WarmStartNet, data, feats, iters=3000, batch=16, lr=2e-3, lr_min=2e-5, seed=0,
          log_every=100):
    """Adam with a cosine learning-rate schedule on random minibatches."""
    import torch
    rng = np.random.default_rng(seed)
    count = data.shape[0]
    losses = []
    for it in range(iters):
        idx = rng.choice(count, size=min(batch, count), replace=False)
        tgt = data.index_select(0, torch.from_numpy(idx).to(data.device))
        y = net.forward(feats[idx])
        part, dy = net.mse(y, tgt)
        net.backward(dy)
        net.adam(lr=lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / iters)))
        if it % log_every == 0 or it == iters - 1:
            losses.append((it, part.sum().item() / y.numel()))
    return losses


def warm_start(net: WarmStartNet, solver, Ra, Pr=0.71, a=DEFAULT_A, buf=None):
    """Initialise a solver (or batch member) from the network's prediction."""
    lib = load_library()
    ny, nx = solver.shape
    if (ny, nx) != (net.size, net.size):
        raise ValueError(f"network predicts {net.size}^2 fields, solver has {nx}x{ny}")
    nodes = nx * ny
    buf = buf or _FieldBuffers(nodes)
    y = net.forward(features([math.log10(Ra)], [Pr], [a]), keep=False)
    T_mid, T_scale, u_scale = _scales(solver.info)
    _ck(lib.islbm_cnn_unpack_fields(ctypes.c_void_p(y.data_ptr()), nodes, T_mid, T_scale,
                                    u_scale, ctypes.c_void_p(buf.T.data_ptr()),
                                    ctypes.c_void_p(buf.u.data_ptr()),
                                    ctypes.c_void_p(buf.v.data_ptr()), _stream()))
    islbm_set_fields_device(solver.h, buf.T, buf.u, buf.v)
    return buf


def compare(net: WarmStartNet, ras, tol=2e-4, sample=1000, window=100, max_steps=4_000_000,
            n=DEFAULT_N, a=DEFAULT_A, pr=0.71, arms=(("fp32", "rest"), ("fp32", "warm"))):
    """Runs of the same cavities to a steady Nu, one batch per arm.

    An arm is (storage precision, start): "rest" is the rest state, "warm" the
    network's prediction.  The criterion is islbm_batch_run_to_steady_nu
    (window means of the volume-averaged Nu, `window` samples `sample` steps
    apart, agreeing to `tol`): on a 256^2 mesh the flow above Ra ~ 3e7 keeps a
    small oscillation and never meets the field criterion.  An arm's wall time
    runs from just after its batch is created (for "warm" it includes the
    network's inference and the equilibrium initialisation) until every cavity
    is steady.  The warm arms also report Nu / Re of the predicted state."""
    import torch
    out = {}
    for precision, start in arms:
        batch = Batch(cavities(ras, n, a, pr), precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if start == "warm":
            buf = _FieldBuffers(n * n)
            for m, r in zip(batch.members, ras):
                warm_start(net, m, r, pr, a, buf)
                m.synchronize()
        steps, nu, re, st = batch.run_to_steady_nu(tol, sample, window, max_steps, check=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        arm = {"precision": precision, "start": start, "steps": list(steps), "status": int(st),
               "wall_s": wall, "Nu": list(nu), "Re": list(re)}
        batch.close()
        if start == "warm":
            probe = Batch(cavities(ras, n, a, pr), precision)
            buf = _FieldBuffers(n * n)
            red0 = []
            for m, r in zip(probe.members, ras):
                warm_start(net, m, r, pr, a, buf)
                red0.append(m.reduce())
            arm["Nu_pred"] = [x["Nu"] for x in red0]
            arm["Re_pred"] = [x["Re"] for x in red0]
            probe.close()
        out[f"{precision}/{start}"] = arm
    return out


def save(net: WarmStartNet, path, meta=None):
    """Weights as stored for inference: matrices in BF16 (the GEMM operands), biases FP32."""
    import torch
    arrays = {}
    for name, w in net.numpy_params().items():
        if name.startswith("W"):
            bits = torch.from_numpy(np.ascontiguousarray(w)).to(torch.bfloat16).view(torch.int16)
            arrays[name] = bits.numpy().view(np.uint16)
        else:
            arrays[name] = np.asarray(w, dtype=np.float32)
    arch = {"base": net.base, "channels": list(net.channels), "hidden": net.hidden,
            "out_ch": net.out_ch}
    np.savez_compressed(path, __arch__=np.frombuffer(repr(arch).encode(), dtype=np.uint8),
                        __meta__=np.frombuffer(repr(meta or {}).encode(), dtype=np.uint8), **arrays)


def load(path, device="cuda") -> WarmStartNet:
    import ast

    import torch
    z = np.load(path)
    arch = ast.literal_eval(bytes(z["__arch__"]).decode())
    net = WarmStartNet(base=arch["base"], channels=tuple(arch["channels"]), hidden=arch["hidden"],
                       out_ch=arch["out_ch"], device=device)
    params = {}
    for name in net.names:
        a = z[name]
        if a.dtype == np.uint16:
            a = torch.from_numpy(a.view(np.int16)).view(torch.bfloat16).to(torch.float32).numpy()
        params[name] = a
    net.load_numpy_params(params)
    return net


def load_meta(path):
    import ast
    return ast.literal_eval(bytes(np.load(path)["__meta__"]).decode())


def main(argv=None):
    """Command line: train (snapshots + training + save) or compare (A/B on held-out Ra).

    Training Ra are log-uniform in [1e6, 1e8] with seed 1, held-out Ra with
    seed 2 (PCG64 draws of the seeded input generators)."""
    import argparse
    import json

    import torch
    from synthetic import ra_sweep

    ap = argparse.ArgumentParser(prog="python -m paper_2509_01099_gb300.warmstart")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--out", required=True)
    tr.add_argument("--cases", type=int, default=100)
    tr.add_argument("--snapshots", type=int, default=20)
    tr.add_argument("--steps", type=int, default=2_000_000)
    tr.add_argument("--every", type=int, default=50_000)
    tr.add_argument("--iters", type=int, default=16000)
    tr.add_argument("--batch", type=int, default=16)
    tr.add_argument("--lr", type=float, default=2e-3)
    tr.add_argument("--log10-lo", type=float, default=6.0)
    tr.add_argument("--log10-hi", type=float, default=8.0)
    ev = sub.add_parser("compare")
    ev.add_argument("--weights", required=True)
    ev.add_argument("--held", type=int, default=16)
    ev.add_argument("--tol", type=float, default=2e-4)
    ev.add_argument("--sample", type=int, default=1000)
    ev.add_argument("--window", type=int, default=100)
    ev.add_argument("--max-steps", type=int, default=4_000_000)
    ev.add_argument("--arms", default="fp32/rest,fp32/warm",
                    help="comma-separated precision/start pairs (start: rest or warm)")
    ev.add_argument("--log10-lo", type=float, default=6.0)
    ev.add_argument("--log10-hi", type=float, default=8.0)
    args = ap.parse_args(argv)

    if args.cmd == "train":
        ras = ra_sweep(args.cases, seed=1, log10_lo=args.log10_lo, log10_hi=args.log10_hi)[0]
        data, feats, glog = snapshot_dataset(ras, args.steps, args.snapshots, args.every)
        print(json.dumps({"snapshots": int(data.shape[0]), "generate_s": glog["wall_s"],
                          "du_last_max": max(glog["du"]) if glog["du"] else None}), flush=True)
        net = WarmStartNet()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = train(net, data, feats, iters=args.iters, batch=args.batch, lr=args.lr)
        torch.cuda.synchronize()
        meta = {"cases": args.cases, "snapshots": int(data.shape[0]), "steps": args.steps,
                "every": args.every, "iters": args.iters, "batch": args.batch,
                "train_s": time.perf_counter() - t0, "loss_first": losses[0][1],
                "loss_last": losses[-1][1], "params": net.n_params,
                "loss_curve": [[int(i), float(v)] for i, v in losses[::10]],
                "log10_ra": [args.log10_lo, args.log10_hi]}
        save(net, args.out, meta)
        print(json.dumps(meta), flush=True)
    else:
        net = load(args.weights)
        ras = ra_sweep(args.held, seed=2, log10_lo=args.log10_lo, log10_hi=args.log10_hi)[0]
        arms = [tuple(x.split("/")) for x in args.arms.split(",")]
        res = compare(net, ras, args.tol, args.sample, args.window, args.max_steps, arms=arms)
        res["Ra"] = [float(r) for r in ras]
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()

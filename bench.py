#!/usr/bin/env python3
"""Benchmark of the fused ISLBM time step on GB300.

Workload (default): the 2-D side-heated cavity at Ra = 1e8, Pr = 0.71 on a
1024 x 1024 tanh-stretched mesh (a = 1.5), D2Q9 + D2Q5, FP32 population
storage.  One bench step is one full ISLBM time step of the whole cavity
(virtual streaming + quadratic interpolation + walls + MRT collision, one fused
kernel).  The timed region holds exactly K steps; before each timed step a
256 MB buffer is written to flush the 126 MB L2 (and a second one read, so
the flush's own dirty lines are written back before the step), and each step is bracketed
by CUDA events on the solver's stream.  The JSON line reports MLUPS
(node updates per second / 1e6), the roofline of the step kernel against the
measured HBM bandwidth, an end-to-end number through the C ABI with host
buffers, and the FP64 oracle timed on the host cores as a CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ISLBM MLUPS & %HBM roofline; wall time to steady Nu, plain vs mixed/learned"
WORKLOAD = "2-D side-heated cavity, D2Q9+D2Q5, Ra=1e8, Pr=0.71, 1024x1024 tanh-stretched mesh (a=1.5)"
BYTES_PER_VALUE = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16dev": "f16", "bf16dev": "bf16"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3],
                    help="2: n x n cavity (D2Q9 + D2Q5); 3: n^3 cavity (D3Q19 + D3Q7)")
    ap.add_argument("--Ra", type=float, default=None,
                    help="Rayleigh number (default: 1e8 in 2-D, 1e7 in 3-D)")
    ap.add_argument("--mesh", default="tanh", choices=["tanh", "erf", "uniform"])
    ap.add_argument("--precision", default="fp32", choices=list(BYTES_PER_VALUE))
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default="auto", help="step-kernel variant (library default: auto)")
    ap.add_argument("--sweep", action="store_true",
                    help="time every kernel variant and storage type; print one JSON line each")
    ap.add_argument("--steady", action="store_true",
                    help="wall time to a steady Nu: plain, mixed precision, learned warm start")
    ap.add_argument("--sweep3d", action="store_true", help="time the 3-D step (256^3)")
    ap.add_argument("--convergence", action="store_true",
                    help="Ra=1e6 grid convergence on 257/513/1025 erf meshes (Table 2)")
    ap.add_argument("--max-steps", type=int, default=0,
                    help="step budget of --convergence / --batch-steady")
    ap.add_argument("--paper-scale", action="store_true",
                    help="the paper's timing workloads: 8193^2 and 400^3, a = 2.1, WCTpDT")
    ap.add_argument("--validate2d", action="store_true",
                    help="2-D cavity at Ra=1e8 to steady state against Table 2's 513^2 row")
    ap.add_argument("--diagnostics", action="store_true",
                    help="boundary layers, their Ra scaling and the divergence of steady cavities")
    ap.add_argument("--validate3d", action="store_true",
                    help="3-D cavity to steady state against the paper's 3-D table (129^3, Ra=1e5)")
    ap.add_argument("--batch-steady", action="store_true",
                    help="the 64-cavity sweep to a steady Nu: batch vs a costed sequential loop")
    ap.add_argument("--series", action="store_true",
                    help="1024^2 Ra=1e8 for --series-steps steps with Nu every 1000 steps")
    ap.add_argument("--series-steps", type=int, default=200_000)
    ap.add_argument("--batch", action="store_true",
                    help="64-cavity Ra sweep: batched persistent launch vs a per-cavity loop")
    args = ap.parse_args()
    if args.Ra is None:
        args.Ra = 1e8 if args.dim == 2 else 1e7
    return args


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


KERNEL_SOURCES = {
    2: ("islbm_d2.cu", "islbm_lanes.cuh", "islbm_store.cuh", "islbm_tma.cuh"),
    3: ("islbm_d3_tma.cu", "islbm_d3_common.cuh", "islbm_lanes.cuh", "islbm_store.cuh",
        "islbm_tma.cuh"),
}


def kernel_source_sha(dim):
    """sha256 over the step kernel's source files (in the order of KERNEL_SOURCES)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[dim]:
        with open(os.path.join(ROOT, "paper_2509_01099_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_traffic(dim, precision, mesh, n):
    """ncu DRAM bytes per launch of the step kernel from the committed summary
    profiles/step{dim}d_{precision}_{mesh}{m}.md taken from the current kernel
    source (else None).  A summary of another size m is scaled by the node
    count (every node's populations are read and written once per step)."""
    import glob
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", f"step{dim}d_{precision}_{mesh}*.md")))
    exact = os.path.join(ROOT, "profiles", f"step{dim}d_{precision}_{mesh}{n}.md")
    if exact in paths:
        paths = [exact]
    for path in paths:
        try:
            text = open(path).read()
            vals = {}
            for line in text.splitlines():
                line = line.strip().lstrip("-").strip()
                if line.startswith(("traffic_bytes_per_launch:", "source_sha256:",
                                    "nodes_per_launch:")):
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.split()[0].strip("`")
            if vals.get("source_sha256") != kernel_source_sha(dim):
                continue
            traffic = float(vals["traffic_bytes_per_launch"])
            if path == exact:
                return traffic
            # another size: only a summary that states its node count (and so
            # claims traffic in proportion to the nodes) is scaled
            if "nodes_per_launch" not in vals:
                continue
            return traffic * (n ** dim) / float(vals["nodes_per_launch"])
        except Exception:
            continue
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_baseline(n: int, steps: int, mesh: str):
    """FP64 numpy oracle on the host cores (one thread), a bounded sample of the workload."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import islbm_oracle as O
from synthetic import temperature_noise
xi = getattr(O, 'mesh_{mesh}')({n}, 1.5) if '{mesh}' != 'uniform' else O.mesh_uniform({n})
cav = O.Cavity(xi, xi, params=O.Params(Ra=1e8))
cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
cav.step(1)
t = time.perf_counter(); cav.step({steps}); dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    return {"value": n * n * steps / (sec * 1e6), "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} time steps of the {n}x{n} {mesh} cavity (Ra=1e8) by the FP64 "
                      f"numpy oracle on one host core ({sec:.1f} s)"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, each step a bounded sample
    (one time step of a 128 x 128 cavity with the workload's mesh and Ra)."""
    if rank != 0:
        return
    from oracle import islbm_oracle as O
    from synthetic import temperature_noise
    n = 128
    xi = O.mesh_uniform(n) if args.mesh == "uniform" else getattr(O, "mesh_" + args.mesh)(n, 1.5)
    cav = O.Cavity(xi, xi, params=O.Params(Ra=args.Ra))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(max(3, args.warmup))
    t = time.perf_counter()
    cav.step(args.steps)
    sec = time.perf_counter() - t
    value = n * n * args.steps / (sec * 1e6)
    sample = f"{args.steps} time steps of a {n}x{n} {args.mesh} cavity (Ra={args.Ra:g}) by the FP64 numpy oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_solver(pkg, n, mesh, Ra, precision, kernel="auto", dim=2):
    """A solver built entirely by the library (its own mesh helpers)."""
    xi = pkg.islbm_mesh_uniform(n) if mesh == "uniform" else getattr(pkg, "islbm_mesh_" + mesh)(n, 1.5)
    return pkg.Solver(*([xi] * dim), Ra=Ra, precision=precision, kernel=kernel)


KERNEL_NAMES = {1: "k_step / k_step3 (direct: one thread per node, interpolation through L1)",
                2: "k_step_tiled (cp.async tile staging)",
                3: "k_step_tma<S,4,2>", 4: "k_step_tma<S,2,2>", 5: "k_step_tma<S,2,3>",
                6: "k_step_tma<S,4,3>",
                7: "k_step3_tma (3-D: warp-specialised TMA ring of population pairs)"}


def sweep(args, pkg, torch, flush):
    """Every step-kernel variant x storage type on the stretched mesh (and the
    direct kernel on the uniform mesh), at n and at 4096^2."""
    for n in (args.n, 4096):
        for mesh in ("tanh", "uniform"):
            for prec in ("fp32", "fp16dev", "bf16dev"):
                kernels = (["direct"] if mesh == "uniform" else
                           [k for k in list(pkg.KERNELS)[1:] if k != "tma3d"])
                for kern in kernels:
                    s = make_solver(pkg, n, mesh, args.Ra, prec, kern)
                    steps = min(args.steps, 400 if n <= 2048 else 100)
                    t = timed_steps(pkg, s, steps, 5, flush, torch)
                    nodes = n * n
                    r = s.reduce(check=False)
                    print(json.dumps({"sweep": True, "n": n, "mesh": mesh, "precision": prec,
                                      "kernel": kern, "MLUPS": nodes * steps / (t * 1e6),
                                      "GBps": 2 * 14 * BYTES_PER_VALUE[prec] * nodes / (t / steps) / 1e9,
                                      "us_per_step": 1e6 * t / steps, "status": r["status"]}),
                          flush=True)
                    s.close()


WARMSTART_WEIGHTS = os.path.join(ROOT, "paper_2509_01099_gb300", "weights", "warmstart_tanh256.npz")


def steady(args, pkg, torch):
    """Wall time to a steady Nu on the 256^2 tanh-stretched cavity (a = 1.5) for
    16 held-out Ra log-uniform in [1e6, 1e8] (PCG64 seed 2): plain (FP32 from
    rest), mixed (FP16 / BF16 deviation storage from rest) and learned (FP32 and
    FP16 started from the warm-start network's prediction).  Each arm is one
    batch of the 16 cavities run until every window mean of Nu (100 samples
    1000 steps apart) changes by at most 2e-4 (islbm_batch_run_to_steady_nu)."""
    from paper_2509_01099_gb300 import warmstart as ws
    from synthetic import ra_sweep
    ras = ra_sweep(16, seed=2)[0]
    net = ws.load(WARMSTART_WEIGHTS)
    arms = (("fp32", "rest"), ("fp16dev", "rest"), ("bf16dev", "rest"), ("fp32", "warm"),
            ("fp16dev", "warm"))
    res = ws.compare(net, ras, arms=arms)
    plain = res["fp32/rest"]
    summary = {}
    for key, arm in res.items():
        nu_dev = [abs(a / b - 1) for a, b in zip(arm["Nu"], plain["Nu"])]
        re_dev = [abs(a / b - 1) for a, b in zip(arm["Re"], plain["Re"])]
        summary[key] = {"wall_s": arm["wall_s"], "steps_total": int(sum(arm["steps"])),
                        "steps_max": int(max(arm["steps"])), "converged": arm["status"] == 0,
                        "wall_rel_to_plain": arm["wall_s"] / plain["wall_s"],
                        "max_Nu_dev_from_plain": max(nu_dev), "max_Re_dev_from_plain": max(re_dev)}
    print(json.dumps({"steady": True, "workload": "2-D cavity 256^2 tanh a=1.5, 16 held-out Ra "
                      "in [1e6, 1e8] (seed 2)", "criterion": "Nu window means, 100 x 1000 steps, "
                      "tol 2e-4", "Ra": [float(r) for r in ras], "summary": summary,
                      "arms": res}), flush=True)


def batch(args, pkg, torch):
    """The batched sweep: 64 2-D cavities, Ra log-uniform in [1e6, 1e8] and
    N from {128, 256, 384, 512} (PCG64 seed 0), tanh meshes (a = 1.5), FP32,
    tile shapes from the autotuner.  Device time of K steps of the whole batch
    (one persistent launch per tile shape and step, replayed from CUDA graphs)
    against the same cavities advanced one after the other."""
    from synthetic import ra_sweep, temperature_noise
    ra, ns = ra_sweep(64, seed=0)
    cavs = [dict(n=int(n), mesh="tanh", a=1.5, Ra=float(r)) for r, n in zip(ra, ns)]
    nodes = sum(c["n"] ** 2 for c in cavities_sorted(cavs))
    K = 640
    t0 = time.perf_counter()
    b = pkg.Batch(cavs, precision="fp32", autotune=True)
    t_setup = time.perf_counter() - t0
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    b.step(128)
    b.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(K)
    e1.record(stream)
    b.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    rows = sorted(set(b.tile_rows(k) for k in range(len(cavs))))
    b.close()
    # the same cavities, one solver after the other (each with its default kernel)
    solvers = []
    for k, c in enumerate(cavs):
        xi = pkg.islbm_mesh_tanh(c["n"], 1.5)
        s = pkg.Solver(xi, xi, Ra=c["Ra"], precision="fp32")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=k))
        s.step(128)
        solvers.append(s)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in solvers:
        s.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for s in solvers:
        s.close()
    print(json.dumps({"batch": True, "cavities": len(cavs), "nodes": nodes, "steps": K,
                      "MLUPS_batched": nodes * K / (t_batch * 1e6),
                      "MLUPS_sequential": nodes * K / (t_seq * 1e6),
                      "speedup": t_seq / t_batch, "tile_rows_used": rows,
                      "setup_s_with_autotune": t_setup,
                      "GBps_batched": 112 * nodes * K / t_batch / 1e9}), flush=True)


def convergence(args, pkg, torch):
    """Grid convergence at Ra = 1e6 (Sec. 3, Table 2): error-function meshes
    (a = 1.5) of 257, 513 and 1025 nodes per axis, FP32, run together as one
    batch from rest until each cavity's Nu window means (50 samples 2000 steps
    apart) agree to 1e-6; then the observed order, the extrapolated value and
    the GCI of every quantity, next to the values Table 2 prints."""
    from paper_2509_01099_gb300 import analysis
    Ns = (257, 513, 1025)
    cavs = [dict(n=n, mesh="erf", a=1.5, Ra=1e6) for n in Ns]
    b = pkg.Batch(cavs, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, nu, re, st = b.run_to_steady_nu(tol=1e-6, sample=2000, window=50,
                                           max_steps=args.max_steps or 12_000_000, check=False)
    wall = time.perf_counter() - t0
    rows = {}
    centre = {}
    for n, m in zip(Ns, b.members):
        r = m.reduce()
        f = m.fields()
        c = n // 2
        # T* = T + 1/2 with the cold-wall reference; u*, v* = u / u_f (Table 3 quantities)
        centre[n] = {"T_c": float(f["T"][c, c] + 0.5), "u_c": float(f["u"][c, c] / m.info.u_f),
                     "v_c": float(f["v"][c, c] / m.info.u_f)}
        for k in ("Nu", "Nu_hot", "Nu_middle", "Re"):
            rows.setdefault(k, []).append(r[k])
    for k in ("u_c", "v_c"):
        rows[k] = [centre[n][k] for n in Ns]
    table = analysis.convergence_table({k: tuple(v) for k, v in rows.items()})
    print(json.dumps({"convergence": True, "workload": "2-D cavity Ra=1e6, erf a=1.5, "
                      "257/513/1025, FP32", "steps": steps, "status": int(st), "wall_s": wall,
                      "window_Nu": nu, "window_Re": re, "centre": centre, "table": table}),
          flush=True)
    b.close()


def series(args, pkg, torch):
    """The 1024^2 Ra = 1e8 cavity run for 200,000 steps from rest (tanh and
    uniform meshes, FP32 and FP16 deviation storage) with the reductions every
    1000 steps: throughput of the whole run (CUDA events, no L2 flush: one
    long job) and the Nu series."""
    from synthetic import temperature_noise
    n, total, every = 1024, args.series_steps, 1000
    for mesh in ("tanh", "uniform"):
        for prec in ("fp32", "fp16dev"):
            s = make_solver(pkg, n, mesh, 1e8, prec)
            s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
            nus, res = [], []
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t_dev = 0.0
            for k in range(total // every):
                e0.record(stream)
                s.step(every)
                e1.record(stream)
                r = s.reduce(check=False)          # synchronises
                t_dev += e0.elapsed_time(e1) / 1e3
                nus.append(r["Nu"])
                res.append(r["Re"])
            mlups = n * n * total / (t_dev * 1e6)
            print(json.dumps({"series": True, "n": n, "mesh": mesh, "precision": prec,
                              "kernel": s.info.kernel, "steps": total, "MLUPS": mlups,
                              "wctpdt_s": (n * n / (mlups * 1e6)) * s.info.steps_per_tf,
                              "tf": total / s.info.steps_per_tf, "Nu_every_1000": nus,
                              "Re_every_1000": res, "status": r["status"]}), flush=True)
            s.close()


def batch_steady(args, pkg, torch):
    """The 64-cavity sweep (as --batch) run from rest to a steady Nu (window means
    of 100 samples 1000 steps apart agreeing to 2e-4, 4M-step budget) as one
    batch, with its wall time; the sequential per-cavity loop is costed from
    each mesh size's measured single-cavity step time times that cavity's
    steps to steady (running 64 cavities one after the other to steady would
    take several times the batch's GPU time)."""
    from synthetic import ra_sweep, temperature_noise
    ra, ns = ra_sweep(64, seed=0)
    cavs = [dict(n=int(n), mesh="tanh", a=1.5, Ra=float(r)) for r, n in zip(ra, ns)]
    b = pkg.Batch(cavs, precision="fp32", autotune=True)
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, nu, re, st = b.run_to_steady_nu(tol=2e-4, sample=1000, window=100,
                                           max_steps=args.max_steps or 4_000_000, check=False)
    wall = time.perf_counter() - t0
    b.close()
    # single-cavity step time per mesh size (default kernel, 2000 steps, CUDA events)
    per_step = {}
    stream = torch.cuda.current_stream()
    for n in sorted(set(int(x) for x in ns)):
        s = pkg.Solver(pkg.islbm_mesh_tanh(n, 1.5), pkg.islbm_mesh_tanh(n, 1.5), Ra=1e7,
                       precision="fp32")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
        s.step(200)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(2000)
        e1.record(stream)
        e1.synchronize()
        per_step[n] = e0.elapsed_time(e1) / 1e3 / 2000
        s.close()
    done = [k for k in steps if k > 0]
    seq = sum(per_step[int(n)] * (k if k > 0 else (args.max_steps or 4_000_000))
              for n, k in zip(ns, steps))
    print(json.dumps({"batch_steady": True, "cavities": len(cavs), "status": int(st),
                      "converged": len(done), "wall_s_batch": wall,
                      "wall_s_sequential_costed": seq, "speedup": seq / wall,
                      "steps": steps, "Ra": [float(r) for r in ra], "n": [int(n) for n in ns],
                      "Nu": nu, "Re": re, "single_cavity_s_per_step": per_step}), flush=True)


def validate2d(args, pkg, torch):
    """The 2-D cavity at Ra = 1e8 against Table 2's 513^2 row (erf mesh a = 1.5,
    Pr = 0.71; <Nu> 30.313, Nu_hot 30.3503, Nu_middle 30.3125, <Re> 542.9352),
    FP32, from rest to a steady Nu (window means of 100 samples 1000 steps
    apart agreeing to 1e-5)."""
    from synthetic import temperature_noise
    n, Ra = 513, 1e8
    b = pkg.Batch([dict(n=n, mesh="erf", a=1.5, Ra=Ra)], precision="fp32")
    m = b.members[0]
    m.set_fields(temperature_noise(m.shape, 1e-6, seed=0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, nu, re, st = b.run_to_steady_nu(tol=1e-5, sample=1000, window=100,
                                           max_steps=args.max_steps or 12_000_000, check=False)
    wall = time.perf_counter() - t0
    red = m.reduce(check=False)
    f = m.fields()
    c = n // 2
    uf = m.info.u_f
    print(json.dumps({"validate2d": True, "n": n, "Ra": Ra, "steps": steps[0], "status": int(st),
                      "wall_s": wall, "tf": steps[0] / m.info.steps_per_tf,
                      "window_Nu": nu[0], "window_Re": re[0], "Nu": red["Nu"],
                      "Nu_hot": red["Nu_hot"], "Nu_cold": red["Nu_cold"],
                      "Nu_middle": red["Nu_middle"], "Re": red["Re"],
                      "T_c": float(f["T"][c, c] + 0.5), "u_c": float(f["u"][c, c] / uf),
                      "v_c": float(f["v"][c, c] / uf),
                      "paper_513": {"Nu": 30.313, "Nu_hot": 30.3503, "Nu_middle": 30.3125,
                                    "Re": 542.9352}}), flush=True)
    b.close()


def diagnostics(args, pkg, torch):
    """Post-processing of steady 2-D cavities (Sec. 3): erf meshes (a = 1.5) of
    257^2 at Ra = 1e6 and 513^2 at Ra = 1e7 and 1e8, FP32, run as one batch to a
    steady Nu (window means agreeing to 1e-5); boundary-layer thicknesses at
    the hot wall from the mid-height band 0.4 <= y* <= 0.6 by the 99% and slope
    methods, their Ra exponents (the paper: -0.25 for both at Pr = 0.71), and
    the statistics of the velocity divergence |div* u*|."""
    import numpy as np
    from paper_2509_01099_gb300 import analysis as A
    from synthetic import temperature_noise
    cases = [(257, 1e6), (513, 1e7), (513, 1e8)]
    b = pkg.Batch([dict(n=n, mesh="erf", a=1.5, Ra=ra) for n, ra in cases], precision="fp32")
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    steps, nu, re, st = b.run_to_steady_nu(tol=1e-5, sample=1000, window=100,
                                           max_steps=args.max_steps or 9_000_000, check=False)
    rows = []
    for (n, ra), m, k in zip(cases, b.members, steps):
        f = m.fields()
        x = A.node_positions(pkg.islbm_mesh_erf(n, 1.5))
        uf = m.info.u_f
        Ts, us, vs = f["T"] + 0.5, f["u"] / uf, f["v"] / uf
        Tb = A.band_profiles(Ts, x)
        vb = A.band_profiles(vs, x)
        bl = A.boundary_layers(x, Tb, vb)
        div = np.abs(A.divergence_2d(us, vs, x, x))
        rows.append({"n": n, "Ra": ra, "steps": k, **bl,
                     "div_median": float(np.median(div)), "div_p99": float(np.percentile(div, 99)),
                     "div_frac_below_1e-4": float((div < 1e-4).mean())})
    ras = [r["Ra"] for r in rows]
    fits = {key: A.power_law(ras, [r[key] for r in rows])[0]
            for key in ("delta_T_99", "delta_V_99", "delta_T_slope", "delta_V_slope")}
    print(json.dumps({"diagnostics": True, "status": int(st), "rows": rows,
                      "exponents": fits, "paper_exponents": {"delta_T": -0.25, "delta_V": -0.25}}),
          flush=True)
    b.close()


def validate3d(args, pkg, torch):
    """The 3-D cavity against Table 3 of the paper's 3-D section (erf mesh, a =
    1.5, Pr = 0.71): 129^3 at Ra = 1e5 (and 181^3 at Ra = 1e6 with --n 181), FP32,
    from rest to the steady criterion of Sec. 3 at 1e-6 over 2000 steps."""
    from synthetic import temperature_noise
    cases = [(129, 1e5)] if args.n != 181 else [(181, 1e6)]
    for n, Ra in cases:
        xi = pkg.islbm_mesh_erf(n, 1.5)
        s = pkg.Solver(xi, xi, xi, Ra=Ra, precision="fp32")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.run_to_steady(tol=1e-6, interval=2000, max_steps=args.max_steps or 3_000_000,
                            check=False)
        wall = time.perf_counter() - t0
        red = s.reduce(check=False)
        f = s.fields()
        c = n // 2
        uf = s.info.u_f
        print(json.dumps({"validate3d": True, "n": n, "Ra": Ra, "kernel": s.info.kernel,
                          "steps": r["steps"], "status": r["status"], "wall_s": wall,
                          "tf": r["steps"] / s.info.steps_per_tf,
                          "Nu": red["Nu"], "Nu_hot": red["Nu_hot"], "Nu_cold": red["Nu_cold"],
                          "Re_rms_uvw": red["Re"], "Re_rms_uv": red["Re_uv"],
                          "Re_mean": red["Re_mean"],
                          "T_c": float(f["T"][c, c, c] + 0.5), "u_c": float(f["u"][c, c, c] / uf),
                          "v_c": float(f["v"][c, c, c] / uf), "w_c": float(f["w"][c, c, c] / uf)}),
              flush=True)
        s.close()


def paper_scale(args, pkg, torch, flush):
    """The paper's own timing workloads (Sec. 3 and the 3-D performance
    paragraph): the 2-D cavity on an 8193^2 error-function mesh with a = 2.1 at
    Ra = 1e8, and the 3-D cavity on a 400^3 mesh with a = 2.1 at Ra = 1e7, in
    FP64 (the paper's precision), FP32 and 16-bit storage; MLUPS and WCTpDT
    (wall-clock seconds per free-fall time), next to the paper's A100 FP64
    WCTpDT of 1.5722e4 s and 1.456e3 s."""
    from synthetic import temperature_noise
    paper = {2: 1.5722e4, 3: 1.456e3}
    for dim, n, Ra in ((2, 8193, 1e8), (3, 400, 1e7)):
        xi = pkg.islbm_mesh_erf(n, 2.1)
        for prec in ("fp64", "fp32", "fp16dev" if dim == 2 else "bf16dev"):
            s = pkg.Solver(*([xi] * dim), Ra=Ra, precision=prec)
            steps = 10 if dim == 3 or prec == "fp64" else 20
            t = timed_steps(pkg, s, steps, 3, flush, torch)
            nodes = n ** dim
            mlups = nodes * steps / (t * 1e6)
            wct = (t / steps) * s.info.steps_per_tf
            print(json.dumps({"paper_scale": True, "dim": dim, "n": n, "a": 2.1, "Ra": Ra,
                              "precision": prec, "kernel": s.info.kernel, "MLUPS": mlups,
                              "wctpdt_s": wct, "steps_per_tf": s.info.steps_per_tf,
                              "paper_wctpdt_s_a100_fp64": paper[dim],
                              "speedup_vs_paper": paper[dim] / wct}), flush=True)
            s.close()


def cavities_sorted(cavs):
    return sorted(cavs, key=lambda c: c["n"])


def sweep3d(args, pkg, torch, flush):
    """The 3-D step (D3Q19 + D3Q7) on the 256^3 tanh mesh and the uniform mesh,
    with the direct kernel and the pipelined TMA kernel."""
    n = 256
    for mesh in ("tanh", "uniform"):
        for prec in ("fp32", "fp16dev", "bf16dev"):
            for kernel in ("direct", "tma3d"):
                xi = pkg.islbm_mesh_uniform(n) if mesh == "uniform" else pkg.islbm_mesh_tanh(n, 1.5)
                s = pkg.Solver(xi, xi, xi, Ra=1e7, precision=prec, kernel=kernel)
                steps = 20
                t = timed_steps(pkg, s, steps, 3, flush, torch)
                nodes = n ** 3
                b = 2 * 26 * BYTES_PER_VALUE[prec]
                print(json.dumps({"sweep3d": True, "n": n, "mesh": mesh, "precision": prec,
                                  "kernel": s.info.kernel, "MLUPS": nodes * steps / (t * 1e6),
                                  "GBps": b * nodes / (t / steps) / 1e9,
                                  "us_per_step": 1e6 * t / steps}), flush=True)
                s.close()


def flush_l2(flush):
    """Write a 256 MB buffer (evicts everything the previous step left in the
    126 MB L2), then read a second 256 MB buffer, so the write-backs of the
    flush itself happen here and the timed step starts on a cold, clean L2."""
    flush[0].zero_()
    flush[1].sum()


def timed_steps(pkg, solver, steps, warmup, flush, torch):
    """Device time of `steps` single-step launches, each after an L2 flush."""
    from synthetic import temperature_noise
    solver.set_fields(temperature_noise(solver.shape, 1e-6, seed=0))
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush_l2(flush)
        solver.step(1)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush_l2(flush)
        starts[k].record(stream)
        solver.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    from paper_2509_01099_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(world)
    if world > 1:
        B.build()
    import paper_2509_01099_gb300 as pkg
    from synthetic import temperature_noise

    n = args.n
    dim = args.dim
    nodes = n ** dim
    flush = [torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda"),
             torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")]
    if args.sweep:
        sweep(args, pkg, torch, flush)
        return
    if args.steady:
        steady(args, pkg, torch)
        return
    if args.sweep3d:
        sweep3d(args, pkg, torch, flush)
        return
    if args.paper_scale:
        paper_scale(args, pkg, torch, flush)
        return
    if args.validate2d:
        validate2d(args, pkg, torch)
        return
    if args.diagnostics:
        diagnostics(args, pkg, torch)
        return
    if args.validate3d:
        validate3d(args, pkg, torch)
        return
    if args.batch_steady:
        batch_steady(args, pkg, torch)
        return
    if args.convergence:
        convergence(args, pkg, torch)
        return
    if args.series:
        series(args, pkg, torch)
        return
    if args.batch:
        batch(args, pkg, torch)
        return
    solver = make_solver(pkg, n, args.mesh, args.Ra, args.precision, args.kernel, dim)
    info = solver.info

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_dev = timed_steps(pkg, solver, args.steps, args.warmup, flush, torch)
    clk = clocks.stop()
    barrier(world)
    t_dev = max_over_ranks(world, t_dev)
    red = solver.reduce(check=False)

    ms_per_step = 1e3 * t_dev / args.steps
    value = world * nodes * args.steps / (t_dev * 1e6)
    bytes_per_update = 2 * (info.q_flow + info.q_temp) * BYTES_PER_VALUE[args.precision]
    achieved = bytes_per_update * nodes / (t_dev / args.steps) / 1e9
    pk = peaks()
    peak, peak_src = (pk["hbm_gbs"], "measured") if pk else (6800.0, "fallback")

    # ---- end to end through the C ABI with host buffers ----
    inner = 100
    pin = lambda: torch.empty(nodes, dtype=torch.float64, pin_memory=True).numpy()
    hT, hu, hv = pin(), pin(), pin()
    hw = pin() if dim == 3 else None
    hT[:] = temperature_noise(solver.shape, 1e-6, seed=0).ravel()
    hu[:] = 0.0
    hv[:] = 0.0
    if hw is not None:
        hw[:] = 0.0
    e2e_iters = max(3, min(20, args.steps // inner))
    solver.set_fields(hT, hu, hv, hw)
    solver.step(inner)
    solver.reduce(check=False)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        solver.set_fields(hT, hu, hv, hw)    # H2D of the step's inputs (pinned)
        solver.step(inner)
        solver.reduce(check=False)           # D2H of the result (Nu, Re, mass, ...)
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = world * nodes * inner * e2e_iters / (t_e2e * 1e6)

    variants = {}
    if not args.no_variants and dim == 2:
        for mesh, prec in (("uniform", "fp32"), ("tanh", "fp16dev"), ("uniform", "fp16dev"),
                           ("tanh", "bf16dev")):
            s2 = make_solver(pkg, n, mesh, args.Ra, prec)
            t2 = timed_steps(pkg, s2, min(args.steps, 500), 10, flush, torch)
            k = min(args.steps, 500)
            b2 = 2 * 14 * BYTES_PER_VALUE[prec]
            variants[f"{mesh}_{prec}"] = {
                "MLUPS": nodes * k / (t2 * 1e6),
                "GBps": b2 * nodes / (t2 / k) / 1e9,
                "ms_per_step": 1e3 * t2 / k}
            s2.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": WORKLOAD if (n == 1024 and args.mesh == "tanh" and dim == 2) else
                       (f"2-D cavity {n}x{n} {args.mesh}, Ra={args.Ra:g}" if dim == 2 else
                        f"3-D cavity {n}^3 {args.mesh}, D3Q19+D3Q7, Ra={args.Ra:g}"),
                       "n": n, "mesh": args.mesh, "a": 1.5, "Ra": args.Ra, "Pr": 0.71,
                       "precision": args.precision, "parallelism": f"replicas{world}",
                       "l2": "before every timed step: 256 MB write, then 256 MB read of another buffer (cold, clean L2)",
                       "L_lu": info.L, "steps_per_tf": info.steps_per_tf},
            "wctpdt_s": ms_per_step * 1e-3 * info.steps_per_tf,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": profile_traffic(dim, args.precision, args.mesh, n),
                         "bytes_per_update": bytes_per_update,
                         "kernel": KERNEL_NAMES.get(info.kernel, str(info.kernel))},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": (dim + 1) * 8 * nodes, "d2h_bytes_per_step": 8 * 16,
                    "definition": f"per step: set_fields from pinned host T,u,v + {inner} time steps + reduce read back"},
            "gpu_launches": args.steps,
            "clocks": clk,
            "state_check": {"Nu": red.get("Nu"), "Re": red.get("Re"), "status": red.get("status")},
            "variants": variants,
        }
        if not args.no_cpu_baseline and dim == 2:
            line["cpu_baseline"] = cpu_baseline(n, 6, args.mesh)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

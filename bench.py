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
BYTES_PER_VALUE = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2, "fp16neq": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16dev": "f16", "bf16dev": "bf16", "fp16neq": "f32+f16"}


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
    ap.add_argument("--steady-precision", action="store_true",
                    help="wall time to a steady Nu of single cavities in FP64 (the paper's "
                         "precision), FP32, FP16NEQ and BF16DEV storage")
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
    ap.add_argument("--timed-sequential", action="store_true",
                    help="with --batch-steady: also run the 64 cavities one after the other to "
                         "a steady Nu and time that loop")
    ap.add_argument("--series", action="store_true",
                    help="1024^2 Ra=1e8 for --series-steps steps with Nu every 1000 steps")
    ap.add_argument("--series-steps", type=int, default=200_000)
    ap.add_argument("--grid-study", action="store_true",
                    help="steady runs on a sequence of erf meshes (--grids, --dim, --Ra), each "
                         "started from the previous one's steady state; observed orders, "
                         "extrapolated values and GCI beside the paper's tables")
    ap.add_argument("--min-steps", type=int, default=0,
                    help="--grid-study: steps every mesh started from a coarser one runs "
                         "before its steady criterion is tested")
    ap.add_argument("--grids", default="513,1025,2049",
                    help="mesh sizes of --grid-study, coarse to fine")
    ap.add_argument("--batch", action="store_true",
                    help="64-cavity Ra sweep: batched persistent launch vs a per-cavity loop")
    ap.add_argument("--cnn-gemm", action="store_true",
                    help="the warm-start network's GEMM shapes (batch 16) on the tcgen05 and "
                         "mma.sync paths: device time, TFLOP/s, GB/s")
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
    3: ("islbm_d3_zm.cu", "islbm_d3_common.cuh", "islbm_lanes.cuh", "islbm_store.cuh",
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


def gpu_selector(local: int) -> str:
    """nvidia-smi -i argument of the GPU this rank runs on.  nvidia-smi numbers
    the physical GPUs and ignores CUDA_VISIBLE_DEVICES, so the device is named
    by its UUID (else its PCI bus id, else the visible-devices entry)."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(local)
        uuid = str(getattr(pr, "uuid", "") or "")
        if uuid:
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        if hasattr(pr, "pci_bus_id"):
            return "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
    except Exception:
        pass
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    return vis[local] if local < len(vis) else str(local)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region,
    of the GPU named by `index` (an nvidia-smi -i selector: UUID, PCI bus id or index)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
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
                "reasons": sorted(reasons), "gpu": str(self.index)}


_ORACLE_SAMPLE = """
import os, sys, time, json
sys.path.insert(0, {root!r})
from oracle import islbm_oracle as O
from synthetic import temperature_noise
xi = getattr(O, 'mesh_{mesh}')({n}, 1.5) if '{mesh}' != 'uniform' else O.mesh_uniform({n})
cav = O.Cavity(xi, xi, params=O.Params(Ra=1e8))
cav.init_fields(temperature_noise(cav.shape, 1e-6, seed={seed}))
cav.step(1)
t = time.perf_counter(); cav.step({steps}); dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt}}))
"""


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(n: int, steps: int, mesh: str):
    """The FP64 numpy oracle on the host cores, a bounded sample of the workload:
    `steps` time steps of the n x n cavity, once on one core, then as one
    independent cavity per core on every core at once (separate processes, one
    BLAS thread each); the all-core rate is the headline value."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cores = os.cpu_count() or 1

    def launch(seed):
        code = _ORACLE_SAMPLE.format(root=ROOT, mesh=mesh, n=n, seed=seed, steps=steps)
        return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                stderr=subprocess.PIPE, text=True, env=env)

    def seconds(proc):
        out, err = proc.communicate(timeout=900)
        if proc.returncode != 0:
            raise RuntimeError(err[-300:])
        return json.loads(out.strip().splitlines()[-1])["seconds"]

    try:
        sec1 = seconds(launch(0))
        t0 = time.perf_counter()
        procs = [launch(k) for k in range(cores)]
        secs = [seconds(p) for p in procs]
        wall = time.perf_counter() - t0
    except Exception as e:   # noqa: BLE001 - reported, not raised
        return {"error": str(e)[-300:]}
    one = n * n * steps / (sec1 * 1e6)
    # aggregate: every core's cavity steps over the slowest core's timed loop
    allc = cores * n * n * steps / (max(secs) * 1e6)
    model = cpu_model()
    return {"value": allc, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} time steps of the {n}x{n} {mesh} cavity (Ra=1e8) by the FP64 "
                      f"numpy oracle, one independent cavity per core on all {cores} cores "
                      f"({model}); slowest core {max(secs):.1f} s, all processes {wall:.1f} s",
            "cpu_model": model,
            "single_core": {"value": one, "unit": "MLUPS", "cores": 1,
                            "sample": f"the same sample on one core ({sec1:.1f} s)"}}


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
    """Reference arm: the FP64 oracle on one host core, each step one time step of
    the workload itself (the n x n cavity with its mesh and Ra; a 3-D workload
    is sampled on a 48^3 cube: the oracle needs ~20 s per step at 256^3)."""
    if rank != 0:
        return
    # one core: numpy's BLAS reads its thread count when it is first imported
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import islbm_oracle as O
    from synthetic import temperature_noise
    n = args.n if args.dim == 2 else 48
    xi = O.mesh_uniform(n) if args.mesh == "uniform" else getattr(O, "mesh_" + args.mesh)(n, 1.5)
    cav = O.Cavity(*([xi] * args.dim), params=O.Params(Ra=args.Ra))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(max(3, args.warmup))
    t = time.perf_counter()
    cav.step(args.steps)
    sec = time.perf_counter() - t
    value = n ** args.dim * args.steps / (sec * 1e6)
    shape = "x".join([str(n)] * args.dim)
    sample = (f"{args.steps} time steps of the {shape} {args.mesh} cavity (Ra={args.Ra:g}) by the "
              f"FP64 numpy oracle on one core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if (args.dim == 2 and args.n == 1024 and
                                                args.mesh == "tanh") else shape + " cavity",
                       "sample": sample},
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
                7: "k_step3_tma (3-D: warp-specialised TMA ring of population pairs)",
                8: "k_step3_zm<S,8> (3-D: z-marching 32x8 columns, TMA rings of levels)",
                9: "k_step3_zm<S,4> (3-D: z-marching 32x4 columns, TMA rings of levels)"}


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
    rest), mixed (FP16 / BF16 deviation storage and FP16 non-equilibrium storage
    from rest) and learned (FP32, FP16 deviations and FP16 non-equilibrium
    storage started from the warm-start network's prediction).  Each arm is one
    batch of the 16 cavities run until every window mean of Nu (100 samples
    1000 steps apart) changes by at most 2e-4 (islbm_batch_run_to_steady_nu)."""
    from paper_2509_01099_gb300 import warmstart as ws
    from synthetic import ra_sweep
    ras = ra_sweep(16, seed=2)[0]
    net = ws.load(WARMSTART_WEIGHTS)
    arms = (("fp32", "rest"), ("fp16dev", "rest"), ("bf16dev", "rest"), ("fp16neq", "rest"),
            ("fp32", "warm"), ("fp16dev", "warm"), ("fp16neq", "warm"))
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


def steady_precision(args, pkg, torch, count=4, tol=2e-4, sample=1000, window=100):
    """Wall time to a steady Nu by storage precision alone: `count` of the 16
    held-out Ra (PCG64 seed 2) of the 256^2 tanh cavity (a = 1.5), each run as
    a single solver from the rest state, one cavity after the other, in FP64
    (the paper's precision), FP32, FP16NEQ and BF16DEV.  The criterion is the
    one of islbm_batch_run_to_steady_nu, applied here on the host: window means
    of Nu over `window` samples `sample` steps apart agreeing to `tol`; the
    step budget is --max-steps per cavity (default 2M).  Deviations are
    relative to the FP64 arm and to the FP32 arm."""
    from synthetic import ra_sweep
    ras = ra_sweep(16, seed=2)[0][:count]
    budget = args.max_steps or 2_000_000
    xi = pkg.islbm_mesh_tanh(256, 1.5)
    res = {}
    for prec in ("fp64", "fp32", "fp16neq", "bf16dev"):
        arm = {"steps": [], "Nu": [], "Re": [], "steady": [], "kernel": None}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ra in ras:
            s = pkg.Solver(xi, xi, Ra=float(ra), precision=prec)
            arm["kernel"] = int(s.info.kernel)
            prev, acc_nu, acc_re, k, t, done = None, 0.0, 0.0, 0, 0, False
            nu = re = float("nan")
            while t + sample <= budget:
                s.step(sample)
                t += sample
                r = s.reduce(check=False)
                acc_nu += r["Nu"]
                acc_re += r["Re"]
                k += 1
                if k < window:
                    continue
                nu, re = acc_nu / window, acc_re / window
                acc_nu = acc_re = 0.0
                k = 0
                if prev is not None and abs(nu - prev) <= tol * abs(nu):
                    done = True
                    break
                prev = nu
            s.close()
            arm["steps"].append(t)
            arm["Nu"].append(nu)
            arm["Re"].append(re)
            arm["steady"].append(done)
        torch.cuda.synchronize()
        arm["wall_s"] = time.perf_counter() - t0
        res[prec] = arm
    out = {"steady_precision": True,
           "workload": "2-D cavity 256^2 tanh a=1.5, Ra: %d of the 16 held-out (seed 2), single "
                       "solvers one after the other from rest" % count,
           "criterion": "Nu window means, %d x %d steps, tol %g; budget %d steps per cavity"
                        % (window, sample, tol, budget),
           "Ra": [float(r) for r in ras], "arms": {}}
    for prec, arm in res.items():
        row = {"wall_s": arm["wall_s"], "steps_total": int(sum(arm["steps"])),
               "all_steady": all(arm["steady"]), "kernel": arm["kernel"],
               "Nu": arm["Nu"], "Re": arm["Re"]}
        for ref in ("fp64", "fp32"):
            b = res[ref]
            row[f"wall_rel_to_{ref}"] = arm["wall_s"] / b["wall_s"]
            row[f"max_Nu_dev_from_{ref}"] = max(abs(x / y - 1) for x, y in zip(arm["Nu"], b["Nu"]))
            row[f"max_Re_dev_from_{ref}"] = max(abs(x / y - 1) for x, y in zip(arm["Re"], b["Re"]))
        out["arms"][prec] = row
    print(json.dumps(out), flush=True)


def steady_lines(pkg, count=4, max_steps=2_000_000):
    """The second half of the metric on a bounded sample: `count` of the 16
    held-out Ra (PCG64 seed 2) of the 256^2 tanh cavity (a = 1.5), each arm one
    batch run to the steady-Nu criterion (window means of 100 samples 1000
    steps apart agreeing to 2e-4): plain FP32 from rest, the learned warm start
    (FP32, including the network's inference), BF16-deviation storage and FP16
    non-equilibrium storage from rest (step budgets capped at `max_steps`).
    Wall times and the largest Nu / Re deviation from the plain arm."""
    from paper_2509_01099_gb300 import warmstart as ws
    from synthetic import ra_sweep
    ras = ra_sweep(16, seed=2)[0][:count]
    net = ws.load(WARMSTART_WEIGHTS)
    res = ws.compare(net, ras, arms=(("fp32", "rest"), ("fp32", "warm"), ("bf16dev", "rest"),
                                     ("fp16neq", "rest")),
                     max_steps=max_steps)
    plain = res["fp32/rest"]
    out = {"Ra": [float(r) for r in ras]}
    for key, name in (("fp32/rest", "plain"), ("fp32/warm", "learned"),
                      ("bf16dev/rest", "mixed_bf16"), ("fp16neq/rest", "mixed_fp16neq")):
        arm = res[key]
        out[name] = {"wall_s": arm["wall_s"], "steps_total": int(sum(arm["steps"])),
                     "all_steady": arm["status"] == 0,
                     "wall_rel_to_plain": arm["wall_s"] / plain["wall_s"],
                     "max_Nu_dev": max(abs(a / b - 1) for a, b in zip(arm["Nu"], plain["Nu"])),
                     "max_Re_dev": max(abs(a / b - 1) for a, b in zip(arm["Re"], plain["Re"]))}
    return out


def batch_measure(pkg, torch, K=640, warm=128):
    """The batched sweep: 64 2-D cavities, Ra log-uniform in [1e6, 1e8] and
    N from {128, 256, 384, 512} (PCG64 seed 0), tanh meshes (a = 1.5), FP32,
    tile shapes from the autotuner.  Device time of K steps of the whole batch
    (one persistent launch per tile shape and step, replayed from CUDA graphs)
    against the same cavities advanced one after the other, K steps each, also
    timed (CUDA events around the whole sequential loop)."""
    from synthetic import ra_sweep, temperature_noise
    ra, ns = ra_sweep(64, seed=0)
    cavs = [dict(n=int(n), mesh="tanh", a=1.5, Ra=float(r)) for r, n in zip(ra, ns)]
    nodes = sum(c["n"] ** 2 for c in cavities_sorted(cavs))
    t0 = time.perf_counter()
    b = pkg.Batch(cavs, precision="fp32", autotune=True)
    t_setup = time.perf_counter() - t0
    for k, m in enumerate(b.members):
        m.set_fields(temperature_noise(m.shape, 1e-6, seed=k))
    b.step(warm)
    b.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(K)
    e1.record(stream)
    b.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    rows = {}
    for k, c in enumerate(cavs):
        rows.setdefault(str(c["n"]), set()).add(b.tile_rows(k))
    rows = {n: sorted(v) for n, v in sorted(rows.items(), key=lambda t: int(t[0]))}
    b.close()
    # the same cavities, one solver after the other (each with its default kernel)
    solvers = []
    for k, c in enumerate(cavs):
        xi = pkg.islbm_mesh_tanh(c["n"], 1.5)
        s = pkg.Solver(xi, xi, Ra=c["Ra"], precision="fp32")
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=k))
        s.step(warm)
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
    peak = (peaks() or {}).get("hbm_gbs", 6800.0)
    return {"cavities": len(cavs), "nodes": nodes, "steps": K,
            "MLUPS": nodes * K / (t_batch * 1e6),
            "MLUPS_sequential_timed": nodes * K / (t_seq * 1e6),
            "speedup_over_sequential": t_seq / t_batch, "tile_rows_by_n": rows,
            "setup_s_with_autotune": t_setup,
            "GBps": 112 * nodes * K / t_batch / 1e9,
            "frac": 112 * nodes * K / t_batch / 1e9 / peak}


def batch(args, pkg, torch):
    print(json.dumps({"batch": True, **batch_measure(pkg, torch)}), flush=True)


def variant(pkg, torch, flush, n, dim, mesh, prec, steps, Ra, peak):
    """One single-cavity line beside the headline: MLUPS, algorithmic GB/s and
    its fraction of the measured copy bandwidth, L2 flushed before every step."""
    s = make_solver(pkg, n, mesh, Ra, prec, dim=dim)
    t = timed_steps(pkg, s, steps, 3, flush, torch)
    info = s.info
    s.close()
    nodes = n ** dim
    b = info.bytes_per_update      # read + write of one node's state (FP16NEQ: 2 x 44 B)
    gbps = b * nodes / (t / steps) / 1e9
    return {"MLUPS": nodes * steps / (t * 1e6), "GBps": gbps, "frac": gbps / peak,
            "ms_per_step": 1e3 * t / steps, "steps": steps,
            "kernel": KERNEL_NAMES.get(info.kernel, str(info.kernel))}


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
    timed = None
    if args.timed_sequential:
        # the same cavities, one at a time, each from the same initial state to
        # the same criterion (a batch of one member: the same kernel and the
        # same steady test)
        seq_steps, seq_nu = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, c in enumerate(cavs):
            b1 = pkg.Batch([c], precision="fp32", autotune=True)
            m1 = b1.members[0]
            m1.set_fields(temperature_noise(m1.shape, 1e-6, seed=k))
            s1, nu1, _, _ = b1.run_to_steady_nu(tol=2e-4, sample=1000, window=100,
                                                max_steps=args.max_steps or 4_000_000,
                                                check=False)
            seq_steps.append(s1[0])
            seq_nu.append(nu1[0])
            b1.close()
        timed = {"wall_s": time.perf_counter() - t0, "steps": seq_steps, "Nu": seq_nu,
                 "same_steps_as_batch": seq_steps == list(steps)}
    print(json.dumps({"batch_steady": True, "cavities": len(cavs), "status": int(st),
                      "converged": len(done), "wall_s_batch": wall,
                      "wall_s_sequential_costed": seq, "speedup": seq / wall,
                      "sequential_timed": timed,
                      "speedup_timed": (timed["wall_s"] / wall) if timed else None,
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


# The paper's steady results (erf meshes, a = 1.5, Pr = 0.71): Table 2 and
# Table 3 (2-D), the 3-D Nusselt / Reynolds table and the 3-D centre-value
# table.  Keys: (dim, Ra) -> {N: values}, plus "inf" and "p" rows.
PAPER_STEADY = {
    (2, 1e6): {257: {"Nu": 8.8282, "Nu_hot": 8.8509, "Nu_middle": 8.8277, "Re": 99.6110},
               513: {"Nu": 8.8202, "Nu_hot": 8.8317, "Nu_middle": 8.8200, "Re": 99.3839},
               1025: {"Nu": 8.8188, "Nu_hot": 8.8246, "Nu_middle": 8.8188, "Re": 99.3576},
               "inf": {"Nu": 8.8186, "Nu_hot": 8.8206, "Nu_middle": 8.8186, "Re": 99.3542},
               "p": {"Nu": 2.6, "Nu_hot": 1.5, "Nu_middle": 2.6, "Re": 3.1}},
    (2, 1e7): {513: {"Nu": 16.5245, "Nu_hot": 16.5461, "Nu_middle": 16.5243, "Re": 230.6601},
               1025: {"Nu": 16.5133, "Nu_hot": 16.5242, "Nu_middle": 16.5133, "Re": 230.2448},
               2049: {"Nu": 16.5114, "Nu_hot": 16.5169, "Nu_middle": 16.5114, "Re": 230.1948},
               "inf": {"Nu": 16.5110, "Nu_hot": 16.5132, "Nu_middle": 16.5110, "Re": 230.1879},
               "p": {"Nu": 2.5, "Nu_hot": 1.6, "Nu_middle": 2.6, "Re": 3.1}},
    (2, 1e8): {513: {"Nu": 30.3130, "Nu_hot": 30.3503, "Nu_middle": 30.3125, "Re": 542.9352},
               1025: {"Nu": 30.2225, "Nu_hot": 30.2423, "Nu_middle": 30.2223, "Re": 537.3420},
               2049: {"Nu": 30.2072, "Nu_hot": 30.2172, "Nu_middle": 30.2072, "Re": 536.6449},
               "inf": {"Nu": 30.2041, "Nu_hot": 30.2096, "Nu_middle": 30.2041, "Re": 536.5456},
               "p": {"Nu": 2.6, "Nu_hot": 2.1, "Nu_middle": 2.6, "Re": 3.0}},
    (3, 1e5): {129: {"Nu": 4.3406, "Nu_hot": 4.3624, "Nu_cold": 4.3624, "Re": 39.4521,
                     "omega_c": 0.2565, "T_c": 0.49948, "u_c": -2.1342e-4, "v_c": 1.3056e-4},
               181: {"Nu": 4.3363, "Nu_hot": 4.3520, "Nu_cold": 4.3520, "Re": 39.3768,
                     "omega_c": 0.2560, "T_c": 0.49949, "u_c": -2.2689e-4, "v_c": 1.2423e-4},
               257: {"Nu": 4.3346, "Nu_hot": 4.3457, "Nu_cold": 4.3457, "Re": 39.3500,
                     "omega_c": 0.2557, "T_c": 0.49950, "u_c": -2.3377e-4, "v_c": 1.2119e-4},
               "inf": {"Nu": 4.3334, "Nu_hot": 4.3362, "Nu_cold": 4.3362, "Re": 39.3352},
               "p": {"Nu": 2.6, "Nu_hot": 1.5, "Nu_cold": 1.5, "Re": 3.0}},
    (3, 1e6): {181: {"Nu": 8.6601, "Nu_hot": 8.6931, "Nu_cold": 8.6931, "Re": 97.4828,
                     "omega_c": 0.1419, "T_c": 0.49942, "u_c": -1.2268e-4, "v_c": 1.4722e-5},
               257: {"Nu": 8.6441, "Nu_hot": 8.6669, "Nu_cold": 8.6668, "Re": 97.0075,
                     "omega_c": 0.1383, "T_c": 0.49946, "u_c": -1.3361e-4, "v_c": 1.6437e-5},
               361: {"Nu": 8.6379, "Nu_hot": 8.6540, "Nu_cold": 8.6540, "Re": 96.8464,
                     "omega_c": 0.1370, "T_c": 0.49948, "u_c": -1.3933e-4, "v_c": 1.7106e-5},
               "inf": {"Nu": 8.6341, "Nu_hot": 8.6419, "Nu_cold": 8.6419, "Re": 96.7638},
               "p": {"Nu": 2.8, "Nu_hot": 2.1, "Nu_cold": 2.1, "Re": 3.1}},
    (3, 1e7): {181: {"Nu": 16.5341, "Nu_hot": 16.6161, "Nu_cold": 16.6158, "Re": 237.3925,
                     "omega_c": 0.1296, "T_c": 0.49898, "u_c": -7.1568e-5, "v_c": 6.1396e-6},
               257: {"Nu": 16.4179, "Nu_hot": 16.4681, "Nu_cold": 16.4680, "Re": 230.7625,
                     "omega_c": 0.1149, "T_c": 0.49917, "u_c": -7.3572e-5, "v_c": 7.4064e-6},
               361: {"Nu": 16.3670, "Nu_hot": 16.4001, "Nu_cold": 16.4001, "Re": 228.4148,
                     "omega_c": 0.1094, "T_c": 0.49926, "u_c": -7.8387e-5, "v_c": 7.7847e-6},
               "inf": {"Nu": 16.3274, "Nu_hot": 16.3422, "Nu_cold": 16.3422, "Re": 227.1278},
               "p": {"Nu": 2.4, "Nu_hot": 2.3, "Nu_cold": 2.3, "Re": 3.0}},
}


def steady_run(pkg, torch, dim, n, Ra, init, tol, max_steps, min_steps=0):
    """One erf-mesh cavity (a = 1.5, FP32) from `init` (None: rest with the seeded
    noise; else fields T, u, v[, w]) to a steady state: in 2-D the Nu-window
    criterion (100 samples 1000 steps apart), then the integral quantities
    averaged over one more such window; in 3-D the field criterion of Sec. 3
    over 2000 steps.  `min_steps` steps run before the criterion is tested (a
    mesh started from a prolongated coarser state can meet the Nu-window
    criterion while its interior still adjusts).  Returns the reductions,
    centre values and fields."""
    import numpy as np
    from paper_2509_01099_gb300 import analysis as A
    from synthetic import temperature_noise
    xi = pkg.islbm_mesh_erf(n, 1.5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if dim == 2:
        b = pkg.Batch([dict(n=n, mesh="erf", a=1.5, Ra=Ra)], precision="fp32")
        s = b.members[0]
    else:
        b = None
        s = pkg.Solver(xi, xi, xi, Ra=Ra, precision="fp32")
    if init is None:
        s.set_fields(temperature_noise(s.shape, 1e-6, seed=0))
    else:
        s.set_fields(init["T"], init["u"], init["v"], init.get("w"))
    pre = min(min_steps, max_steps)
    if pre:
        (b if b is not None else s).step(pre)
    if dim == 2:
        steps, _, _, st = b.run_to_steady_nu(tol=tol, sample=1000, window=100,
                                             max_steps=max_steps - pre, check=False)
        steps = steps[0] + pre
    else:
        r = s.run_to_steady(tol=tol, interval=2000, max_steps=max_steps - pre, check=False)
        steps, st = r["steps"] + pre, r["status"]
    wall = time.perf_counter() - t0
    red = s.reduce(check=False)
    red_inst = dict(red)
    if dim == 2:
        # the integral quantities as means over one more window (100 samples
        # 1000 steps apart): at Ra = 1e8 a small residual oscillation survives
        # the window criterion, and a single sample of <Nu> or Nu_middle can
        # sit on its crest
        keys = ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re", "Re_uv")
        acc = {k: 0.0 for k in keys}
        for _ in range(100):
            b.step(1000)
            r = s.reduce(check=False)
            for k in keys:
                acc[k] += r[k] / 100
        red.update(acc)
        steps += 100_000
    f = s.fields()
    uf = s.info.u_f
    fields = {k: np.asarray(v) for k, v in f.items()}
    if dim == 2:
        c = A.centre_values_2d(xi, xi, f["T"] + 0.5, f["u"] / uf, f["v"] / uf)
    else:
        c = A.centre_values_3d(xi, xi, xi, f["T"] + 0.5, f["u"] / uf, f["v"] / uf, f["w"] / uf)
    out = {"n": n, "steps": int(steps), "status": int(st), "wall_s": wall,
           "tf": steps / s.info.steps_per_tf, "kernel": s.info.kernel,
           "Nu": red["Nu"], "Nu_hot": red["Nu_hot"], "Nu_cold": red["Nu_cold"],
           "Nu_middle": red["Nu_middle"] if dim == 2 else None, "Re": red["Re"],
           "Re_uv": red["Re_uv"], "T_c": c["T"], "u_c": c["u"], "v_c": c["v"],
           "omega_c": abs(c["omega"]),
           "Nu_at_criterion": red_inst["Nu"], "Nu_middle_at_criterion": red_inst["Nu_middle"]}
    if b is not None:
        b.close()
    else:
        s.close()
    return out, {k: fields[k] for k in ("T", "u", "v") + (("w",) if dim == 3 else ())}


def grid_study(args, pkg, torch):
    """Steady cavities on a sequence of erf meshes (a = 1.5), coarse to fine,
    each finer run started from the prolongated steady state of the one before
    (grid sequencing: the transient is not repeated on the fine meshes); the
    observed orders, Richardson-extrapolated values and GCI (Sec. 3) beside the
    paper's rows for the same Ra."""
    import math
    from paper_2509_01099_gb300 import analysis as A
    dim, Ra = args.dim, args.Ra
    grids = [int(g) for g in args.grids.split(",")]
    tol = 1e-6 if dim == 3 else (1e-5 if Ra >= 1e8 else 1e-6)
    rows, prev, prev_n = [], None, None
    for n in grids:
        init = None
        if prev is not None:
            xc = pkg.islbm_mesh_erf(prev_n, 1.5)
            xf = pkg.islbm_mesh_erf(n, 1.5)
            init = A.prolong(prev, [xc] * dim, [xf] * dim)
        row, fields = steady_run(pkg, torch, dim, n, Ra, init, tol,
                                 args.max_steps or (12_000_000 if dim == 2 else 3_000_000),
                                 args.min_steps if init is not None else 0)
        row["started_from"] = prev_n
        rows.append(row)
        print(json.dumps({"grid_study_row": True, "dim": dim, "Ra": Ra, **row}), flush=True)
        prev, prev_n = fields, n
    table = None
    if len(grids) == 3:
        ratio = math.sqrt((grids[2] - 1) / (grids[0] - 1))
        keys = ["Nu", "Nu_hot", "Re"] + (["Nu_middle"] if dim == 2 else ["Nu_cold"]) + \
            ["T_c", "u_c", "v_c", "omega_c"]
        table = A.convergence_table({k: tuple(r[k] for r in rows) for k in keys}, ratio=ratio)
    print(json.dumps({"grid_study": True, "dim": dim, "Ra": Ra, "grids": grids,
                      "criterion": ("Nu window means, 100 x 1000 steps, tol %g" % tol) if dim == 2
                      else ("field change over 2000 steps below %g (Sec. 3)" % tol),
                      "rows": rows, "richardson": table,
                      "paper": {str(k): v for k, v in PAPER_STEADY.get((dim, Ra), {}).items()}}),
          flush=True)


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


def cnn_gemm(pkg, torch, batch=16, reps=20):
    """Device time of the warm-start network's products at batch 16: for every
    convolution of the decoder (16^2 .. 256^2) the forward product (im2col rows
    x weights), the data gradient (dY x W^T) and the weight gradient
    (im2col^T x dY), on path 1 (mma.sync) and path 2 (tcgen05 + TMA, where
    its 16-byte conditions hold), with 3 warm-up calls and `reps` timed ones.
    Algorithmic bytes: the BF16 operands read once and the FP32 result
    written once."""
    import ctypes
    from paper_2509_01099_gb300.islbm import load_library
    lib = load_library()
    st = torch.cuda.current_stream()
    S = ctypes.c_void_p(st.cuda_stream)
    layers = [(16, 64, 64), (32, 64, 48), (64, 48, 32), (128, 32, 16), (256, 16, 16), (256, 16, 3)]
    g = torch.Generator(device="cuda").manual_seed(0)
    for hw, cin, cout in layers:
        M, kp = batch * hw * hw, (9 * cin + 15) // 16 * 16
        for name, m, n, k, ta, tb in ((f"fwd {hw}^2 {cin}->{cout}", M, cout, kp, 0, 0),
                                      (f"dgrad {hw}^2", M, kp, cout, 0, 1),
                                      (f"wgrad {hw}^2", kp, cout, M, 1, 0)):
            A = torch.randn((k, m) if ta else (m, k), device="cuda", generator=g).to(torch.bfloat16)
            B = torch.randn((n, k) if tb else (k, n), device="cuda", generator=g).to(torch.bfloat16)
            C = torch.zeros((m, n), device="cuda")
            row = {"cnn_gemm": name, "M": m, "N": n, "K": k}
            for path in (1, 2):
                if path == 2 and (A.shape[1] % 8 or B.shape[1] % 8):
                    continue
                call = lambda: lib.islbm_cnn_gemm_bf16_ex(
                    ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                    ctypes.c_void_p(C.data_ptr()), None, m, n, k, A.shape[1], B.shape[1], n, ta,
                    tb, 0, path, S)
                for _ in range(3):
                    if call() != 0:
                        raise RuntimeError(f"islbm_cnn_gemm_bf16_ex failed on {name}")
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                for _ in range(reps):
                    call()
                e1.record(st)
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) * 1e3 / reps
                tag = "tcgen05" if path == 2 else "mma_sync"
                row[f"us_{tag}"] = round(us, 2)
                row[f"tflops_{tag}"] = round(2.0 * m * n * k / us / 1e6, 2)
                row[f"gbps_{tag}"] = round((2 * (m * k + k * n) + 4 * m * n) / us / 1e3, 1)
            print(json.dumps(row), flush=True)


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
    if args.cnn_gemm:
        cnn_gemm(pkg, torch)
        return
    if args.steady:
        steady(args, pkg, torch)
        return
    if args.steady_precision:
        steady_precision(args, pkg, torch)
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
    if args.grid_study:
        grid_study(args, pkg, torch)
        return
    solver = make_solver(pkg, n, args.mesh, args.Ra, args.precision, args.kernel, dim)
    info = solver.info

    clocks = ClockSampler(gpu_selector(local))
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
    bytes_per_update = info.bytes_per_update
    achieved = bytes_per_update * nodes / (t_dev / args.steps) / 1e9
    pk = peaks()
    peak, peak_src = (pk["hbm_gbs"], "measured") if pk else (6800.0, "fallback")

    # ---- end to end through the C ABI with host buffers ----
    # One iteration: the initial fields from pinned host memory (equilibrium
    # initialisation), `inner` time steps, the reductions and the fields T, u,
    # v (, w) back to host memory.  Reported per time step: the copies of an
    # iteration divided by its `inner` steps.
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
    hout = {k: pin() for k in ("rho", "T", "u", "v") + (("w",) if dim == 3 else ())}
    solver.set_fields(hT, hu, hv, hw)
    solver.step(inner)
    solver.reduce(check=False)
    solver.fields(out=hout)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        solver.set_fields(hT, hu, hv, hw)    # H2D of the inputs (pinned)
        solver.step(inner)
        solver.reduce(check=False)           # D2H of the reductions (Nu, Re, mass, ...)
        out = solver.fields(out=hout)        # D2H of the fields rho, T, u, v (, w), pinned
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = world * nodes * inner * e2e_iters / (t_e2e * 1e6)
    h2d = (dim + 1) * 8 * nodes
    d2h = 8 * 16 + sum(a.nbytes for a in out.values())

    variants = {}
    if not args.no_variants and dim == 2 and rank == 0:
        k = min(args.steps, 500)
        for mesh, prec in (("uniform", "fp32"), ("tanh", "fp16dev"), ("uniform", "fp16dev"),
                           ("tanh", "bf16dev"), ("tanh", "fp16neq")):
            variants[f"{mesh}_{prec}"] = variant(pkg, torch, flush, n, 2, mesh, prec, k, args.Ra,
                                                 peak)
        # far above L2: the roofline regime (4096^2, 2 x 1.9 GB of FP32 state)
        for prec in ("fp32", "bf16dev", "fp16neq"):
            variants[f"tanh4096_{prec}"] = variant(pkg, torch, flush, 4096, 2, "tanh", prec,
                                                   min(args.steps, 50), args.Ra, peak)
        # the 3-D cavity workload: 256^3 tanh mesh, Ra = 1e7
        for prec in ("fp32", "bf16dev"):
            variants[f"cube256_tanh_{prec}"] = variant(pkg, torch, flush, 256, 3, "tanh", prec,
                                                       min(args.steps, 20), 1e7, peak)
        # the 64-cavity batched sweep against the same cavities stepped one by one
        variants["batch64_fp32"] = batch_measure(pkg, torch, K=64, warm=64)
        # wall time to a steady Nu: plain, learned warm start, mixed precision
        variants["steady_256_4ra"] = steady_lines(pkg)

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
                       "l2_regime": (f"state {bytes_per_update * nodes / 1e6:.0f} MB "
                                     f"(two time levels) against a 126 MB L2: "
                                     + ("reads come from DRAM, but much of what a step writes "
                                        "is still in L2 when it ends; frac is algorithmic bytes "
                                        "over time, the DRAM traffic is in roofline.traffic"
                                        if bytes_per_update * nodes < 2.5e8 else
                                        "far above L2, every step streams from and to DRAM")),
                       "L_lu": info.L, "steps_per_tf": info.steps_per_tf},
            "wctpdt_s": ms_per_step * 1e-3 * info.steps_per_tf,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": profile_traffic(dim, args.precision, args.mesh, n),
                         "bytes_per_update": bytes_per_update,
                         "kernel": KERNEL_NAMES.get(info.kernel, str(info.kernel))},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d / inner, "d2h_bytes_per_step": d2h / inner,
                    "definition": (f"iterations of: set_fields from pinned host T, u, v "
                                   f"({h2d} B), {inner} time steps, the reductions and "
                                   f"get_fields of rho, T, u, v back to the host ({d2h} B); "
                                   f"bytes per time step = per iteration / {inner}")},
            "gpu_launches": args.steps,
            "clocks": clk,
            "state_check": {"Nu": red.get("Nu"), "Re": red.get("Re"), "status": red.get("status")},
            "variants": variants,
        }
        if not args.no_cpu_baseline and dim == 2:
            line["cpu_baseline"] = cpu_baseline(n, 4, args.mesh)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

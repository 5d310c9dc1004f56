"""Named run configurations (JSON-compatible dicts) and their construction.

A configuration names the cavity (dimension, nodes per axis, mesh kind and
stretching), the physics (Ra, Pr), the storage precision and the run length;
`solver_from_config` builds the solver through the C ABI and
`load_config` reads one from a JSON file.  The named entries are the
workloads this library is measured on.
"""
from __future__ import annotations

import json

from .islbm import Solver, islbm_mesh_erf, islbm_mesh_tanh, islbm_mesh_uniform

CONFIGS = {
    # 2-D cavity, Ra = 1e6, 64^2 tanh mesh, FP64, 20,000 steps (parity workload)
    "cavity2d_ra1e6_n64_fp64": {"dim": 2, "n": 64, "mesh": "tanh", "a": 1.5, "Ra": 1e6,
                                "Pr": 0.71, "precision": "fp64", "steps": 20_000},
    # 2-D cavity, Ra = 1e8, 1024^2 tanh mesh, FP32 and FP16 deviations, 200,000 steps
    "cavity2d_ra1e8_n1024_fp32": {"dim": 2, "n": 1024, "mesh": "tanh", "a": 1.5, "Ra": 1e8,
                                  "Pr": 0.71, "precision": "fp32", "steps": 200_000},
    "cavity2d_ra1e8_n1024_fp16dev": {"dim": 2, "n": 1024, "mesh": "tanh", "a": 1.5, "Ra": 1e8,
                                     "Pr": 0.71, "precision": "fp16dev", "steps": 200_000},
    # 3-D cavity, Ra = 1e7, 256^3 tanh mesh, FP32 and BF16 deviations
    "cavity3d_ra1e7_n256_fp32": {"dim": 3, "n": 256, "mesh": "tanh", "a": 1.5, "Ra": 1e7,
                                 "Pr": 0.71, "precision": "fp32", "steps": 1000},
    "cavity3d_ra1e7_n256_bf16dev": {"dim": 3, "n": 256, "mesh": "tanh", "a": 1.5, "Ra": 1e7,
                                    "Pr": 0.71, "precision": "bf16dev", "steps": 1000},
    # validation cases of the paper's tables (error-function mesh)
    "cavity2d_ra1e6_n257_erf": {"dim": 2, "n": 257, "mesh": "erf", "a": 1.5, "Ra": 1e6,
                                "Pr": 0.71, "precision": "fp32", "steps": 1_500_000},
    "cavity3d_ra1e5_n129_erf": {"dim": 3, "n": 129, "mesh": "erf", "a": 1.5, "Ra": 1e5,
                                "Pr": 0.71, "precision": "fp32", "steps": 500_000},
}

REQUIRED = ("dim", "n", "mesh", "Ra")


def validate(cfg: dict) -> dict:
    """Fill defaults and check a configuration; raises ValueError."""
    missing = [k for k in REQUIRED if k not in cfg]
    if missing:
        raise ValueError(f"configuration lacks {missing}")
    out = {"a": 1.5, "Pr": 0.71, "precision": "fp32", "steps": 0, "kernel": "auto"}
    out.update(cfg)
    if out["dim"] not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if out["mesh"] not in ("uniform", "erf", "tanh"):
        raise ValueError("mesh must be uniform, erf or tanh")
    if int(out["n"]) < 4:
        raise ValueError("n must be at least 4")
    if not (out["Ra"] > 0 and out["Pr"] > 0):
        raise ValueError("Ra and Pr must be positive")
    return out


def mesh(cfg: dict):
    """The ghost-node mesh of one axis (library helpers)."""
    n, kind = int(cfg["n"]), cfg["mesh"]
    if kind == "uniform":
        return islbm_mesh_uniform(n)
    return (islbm_mesh_erf if kind == "erf" else islbm_mesh_tanh)(n, float(cfg.get("a", 1.5)))


def load_config(path_or_name) -> dict:
    """A named configuration, or one read from a JSON file."""
    if isinstance(path_or_name, dict):
        return validate(path_or_name)
    if path_or_name in CONFIGS:
        return validate(dict(CONFIGS[path_or_name]))
    with open(path_or_name) as f:
        return validate(json.load(f))


def solver_from_config(cfg, stream=None) -> Solver:
    cfg = load_config(cfg)
    xi = mesh(cfg)
    return Solver(*([xi] * cfg["dim"]), Ra=cfg["Ra"], Pr=cfg["Pr"], precision=cfg["precision"],
                  stream=stream, kernel=cfg["kernel"])

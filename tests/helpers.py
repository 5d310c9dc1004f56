"""Shared helpers of the parity tests (no method arithmetic here)."""
import numpy as np


def rel_field_error(gpu: np.ndarray, ref: np.ndarray) -> float:
    """max |gpu - ref| / max |ref| over the nodes (a field-relative error: u and v
    start at zero, so pointwise relative errors are ill-posed)."""
    scale = np.abs(ref).max()
    return float(np.abs(gpu - ref).max() / scale) if scale > 0 else float(np.abs(gpu - ref).max())


def rel_vector_error(got, ref) -> float:
    """Velocity as one vector field: max over nodes and components of |gpu - ref|,
    divided by the largest speed of the reference field."""
    speed = np.sqrt(sum(np.asarray(r) ** 2 for r in ref)).max()
    diff = max(float(np.abs(np.asarray(g) - np.asarray(r)).max()) for g, r in zip(got, ref))
    return diff / speed if speed > 0 else diff


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False

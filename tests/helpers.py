"""Shared helpers of the parity tests (no method arithmetic here)."""
import numpy as np


def rel_field_error(gpu: np.ndarray, ref: np.ndarray) -> float:
    """max |gpu - ref| / max |ref| over the nodes (a field-relative error: u and v
    start at zero, so pointwise relative errors are ill-posed)."""
    scale = np.abs(ref).max()
    return float(np.abs(gpu - ref).max() / scale) if scale > 0 else float(np.abs(gpu - ref).max())


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False

"""The learned warm start against the unaided solver (GPU).

The committed network (paper_2509_01099_gb300/weights/warmstart_tanh256.npz)
was trained by `python -m paper_2509_01099_gb300.warmstart train` on 2,000
late-time snapshots of 100 cavities (Ra log-uniform in [1e6, 1e8], PCG64
seed 1) generated by the batched solver on the 256^2 tanh mesh (a = 1.5).
Held-out Ra come from seed 2.
"""
import math
import os

import numpy as np
import pytest

from oracle import cnn_oracle as oc
from synthetic import ra_sweep
from tests.helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA device")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2509_01099_gb300", "weights", "warmstart_tanh256.npz")


def _net():
    from paper_2509_01099_gb300 import warmstart as ws
    return ws.load(WEIGHTS)


def test_trained_network_inference_matches_oracle():
    """The trained network through the library's kernels against the float64
    oracle with the same (BF16-stored) weights; tolerance as for the random
    networks of test_cnn_gpu (2e-2 relative, BF16 operands)."""
    from paper_2509_01099_gb300.cnn import features
    net = _net()
    assert net.size == 256 and 1.0e6 < net.n_params < 1.3e6
    z = features(np.log10([1.5e6, 2.0e7, 8.0e7]), [0.71] * 3, [1.5] * 3)
    y = net.forward(z, keep=False).cpu().numpy().astype(np.float64)
    params = {k: v.astype(np.float64) for k, v in net.numpy_params().items()}
    yo, _ = oc.forward(params, z, net.base, len(net.channels))
    err = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert err < 2e-2, err
    # the predicted temperature lies between the wall temperatures and is hotter on the hot side
    T = y[..., 0]
    assert np.all(np.abs(T) < 0.6)
    assert (T[:, :, :8].mean(axis=2) > T[:, :, -8:].mean(axis=2)).all()


def test_warm_start_reaches_the_steady_nu_sooner():
    """Four held-out Ra, FP32, from rest and from the network's prediction, to
    the steady-Nu criterion: the warm start needs at most 60% of the steps and
    less wall time, and both reach the same Nu and Re within 0.5%."""
    from paper_2509_01099_gb300 import warmstart as ws
    net = _net()
    ras = ra_sweep(16, seed=2)[0][:4]
    res = ws.compare(net, ras)
    rest, warm = res["fp32/rest"], res["fp32/warm"]
    assert rest["status"] == 0 and warm["status"] == 0
    assert sum(warm["steps"]) <= 0.6 * sum(rest["steps"]), (rest["steps"], warm["steps"])
    assert warm["wall_s"] < rest["wall_s"]
    for a, b in zip(warm["Nu"], rest["Nu"]):
        assert abs(a / b - 1) < 5e-3, (a, b)
    for a, b in zip(warm["Re"], rest["Re"]):
        assert abs(a / b - 1) < 5e-3, (a, b)
    # the prediction itself is already close to the steady state
    for a, b in zip(warm["Nu_pred"], rest["Nu"]):
        assert abs(a / b - 1) < 0.1
    assert all(math.isfinite(v) for v in warm["Re_pred"])

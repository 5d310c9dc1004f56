"""Pins of the warm-start network's float64 oracle (CPU only).

The network is not in the paper; its oracle is the plain definition of the
layers.  These tests tie it to things other than itself: scipy's 2-D
cross-correlation, central finite differences of the loss, the adjoint
identity of the upsampling, and closed forms of the Adam step.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as cnn
from synthetic import gaussian_arrays


def tiny_net(seed=3, F=4, hidden=5, base=2, channels=(3, 2), out=2):
    shapes = [("W1", (F, hidden)), ("b1", (hidden,)),
              ("W2", (hidden, base * base * channels[0])), ("b2", (base * base * channels[0],))]
    cin = channels[0]
    for s, cout in enumerate(list(channels[1:]) + [out]):
        shapes += [(f"Wc{s}", (9 * cin, cout)), (f"bc{s}", (cout,))]
        cin = cout
    params = gaussian_arrays(shapes, seed, {n: 0.6 for n, _ in shapes})
    return params, base, len(channels)


def test_conv3x3_matches_scipy_correlate2d():
    g = gaussian_arrays([("x", (2, 5, 7, 3)), ("W", (27, 4)), ("b", (4,))], seed=1)
    y = cnn.conv3x3(g["x"], g["W"], g["b"])
    Wt = g["W"].reshape(3, 3, 3, 4)
    for b in range(2):
        for o in range(4):
            ref = sum(correlate2d(g["x"][b, :, :, c], Wt[:, :, c, o], mode="same",
                                  boundary="fill") for c in range(3)) + g["b"][o]
            np.testing.assert_allclose(y[b, :, :, o], ref, rtol=0, atol=1e-13)


def test_up2_adjoint_identity():
    g = gaussian_arrays([("x", (2, 3, 4, 5)), ("y", (2, 6, 8, 5))], seed=2)
    lhs = np.vdot(cnn.up2(g["x"]), g["y"])
    rhs = np.vdot(g["x"], cnn.up2_adjoint(g["y"]))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # nearest neighbour: every 2x2 block repeats its source pixel
    u = cnn.up2(g["x"])
    assert np.array_equal(u[:, 1::2, 0::2], g["x"]) and np.array_equal(u[:, 0::2, 1::2], g["x"])


def _loss(params, z, t, wc, base, n_stages):
    y, _ = cnn.forward(params, z, base, n_stages)
    return cnn.mse(y, t, wc)[0]


def test_gradients_match_central_differences():
    params, base, ns = tiny_net()
    g = gaussian_arrays([("z", (3, 4)), ("t", (3, 4, 4, 2))], seed=4)
    wc = np.array([1.0, 2.5])
    y, cache = cnn.forward(params, g["z"], base, ns)
    assert y.shape == (3, 4, 4, 2)
    _, dy = cnn.mse(y, g["t"], wc)
    grads = cnn.backward(params, cache, dy, ns)
    assert set(grads) == set(params)
    h = 1e-6
    for name, w in params.items():
        flat = w.reshape(-1)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h
            lp = _loss(params, g["z"], g["t"], wc, base, ns)
            flat[k] = old - h
            lm = _loss(params, g["z"], g["t"], wc, base, ns)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[k]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), (name, k, fd, an)


def test_mse_definition_and_zero_at_target():
    g = gaussian_arrays([("y", (2, 3, 3, 3)), ("t", (2, 3, 3, 3))], seed=5)
    loss, dy = cnn.mse(g["y"], g["y"])
    assert loss == 0.0 and not dy.any()
    wc = np.array([1.0, 0.0, 3.0])
    loss, _ = cnn.mse(g["y"], g["t"], wc)
    # channel 1 carries no weight; the other two are a plain weighted mean
    r = g["y"] - g["t"]
    manual = (r[..., 0] ** 2).sum() + 3.0 * (r[..., 2] ** 2).sum()
    assert abs(loss - manual / r.size) < 1e-14 * manual


def test_adam_first_step_is_a_sign_step():
    # at t = 1 the bias-corrected moments are g and g^2: the step is lr g / (|g| + eps)
    g = gaussian_arrays([("w", (50,)), ("g", (50,))], seed=6)
    w1, m, v = cnn.adam(g["w"], g["g"], np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(w1, g["w"] - 0.01 * np.sign(g["g"]), rtol=0, atol=1e-15)


def test_adam_constant_gradient_moves_at_constant_rate():
    # with a constant gradient the bias corrections make m_hat = g, v_hat = g^2 at every t
    g = gaussian_arrays([("w", (20,)), ("g", (20,))], seed=7)
    w, m, v = g["w"].copy(), np.zeros(20), np.zeros(20)
    for t in range(1, 40):
        w, m, v = cnn.adam(w, g["g"], m, v, t, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(w, g["w"] - 39 * 1e-3 * np.sign(g["g"]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("drop", ["tanh_back", "flipped_kernel"])
def test_planted_mistakes_fail_the_difference_check(drop, monkeypatch):
    """A dropped activation derivative or a flipped kernel (convolution for
    cross-correlation) in the backward pass must be caught by the
    finite-difference comparison."""
    params, base, ns = tiny_net(seed=8)
    g = gaussian_arrays([("z", (2, 4)), ("t", (2, 4, 4, 2))], seed=9)
    y, cache = cnn.forward(params, g["z"], base, ns)
    _, dy = cnn.mse(y, g["t"])
    if drop == "tanh_back":
        bad_cache = dict(cache, ys=[np.zeros_like(a) for a in cache["ys"]])
        grads = cnn.backward(params, bad_cache, dy, ns)
        name = "Wc0"
    else:
        orig = cnn.conv3x3_backward

        def flipped(x, W, d):
            dx, dW, db = orig(x, W[::-1].copy(), d)
            return dx, dW, db
        monkeypatch.setattr(cnn, "conv3x3_backward", flipped)
        grads = cnn.backward(params, cache, dy, ns)
        name = "W1"
    flat = params[name].reshape(-1)
    h, worst = 1e-6, 0.0
    for k in range(flat.size):
        old = flat[k]
        flat[k] = old + h
        lp = _loss(params, g["z"], g["t"], None, base, ns)
        flat[k] = old - h
        lm = _loss(params, g["z"], g["t"], None, base, ns)
        flat[k] = old
        worst = max(worst, abs((lp - lm) / (2 * h) - grads[name].reshape(-1)[k]))
    assert worst > 1e-5

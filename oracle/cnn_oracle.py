"""Float64 reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

The paper has no network: this oracle is the plain definition of the small
decoder that predicts a steady cavity state from three scalars, used to check
the CUDA kernels' forward pass, gradients and optimiser step.  Only the tests,
the smoke check and the CPU timing of the benchmark may import it.

Definition (NHWC tensors, parameters in a dict):
    h1 = tanh(z W1 + b1)                      z: [B, F]
    x0 = tanh(h1 W2 + b2) reshaped [B, base, base, C0]
    stage s (all but the last): x_{s+1} = tanh(conv3x3(up2(x_s), Wc_s) + bc_s)
    last stage:                 y       = conv3x3(x_s, Wc_s) + bc_s
up2 repeats every pixel into a 2x2 block (nearest neighbour); conv3x3 is the
zero-padded 'same' cross-correlation
    conv(x, W)[b, i, j, o] = sum_{dy, dx in -1..1} sum_c x[b, i+dy, j+dx, c] W[tap, c, o]
with tap = 3 (dy + 1) + (dx + 1) and Wc_s stored as [9 C_in, C_out] rows
ordered (tap, c).  Loss: weighted mean squared error
    L = (1/n) sum_e w_{c(e)} (y_e - t_e)^2 over all n output values.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def stage_names(n_stages):
    return [(f"Wc{s}", f"bc{s}") for s in range(n_stages)]


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_adjoint(d):
    B, H2, W2, C = d.shape
    return d.reshape(B, H2 // 2, 2, W2 // 2, 2, C).sum(axis=(2, 4))


def conv3x3(x, W, b):
    """Zero-padded 3x3 cross-correlation; W [9 Cin, Cout]."""
    B, H, Wd, C = x.shape
    Wt = W.reshape(3, 3, C, -1)
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((B, H, Wd, Wt.shape[-1]))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bijc,co->bijo", xp[:, dy:dy + H, dx:dx + Wd], Wt[dy, dx])
    return y + b


def conv3x3_backward(x, W, d):
    """Gradients of sum(d * conv3x3(x, W, b)) with respect to x, W and b."""
    B, H, Wd, C = x.shape
    Wt = W.reshape(3, 3, C, -1)
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(Wt)
    for dy in range(3):
        for dx in range(3):
            dW[dy, dx] = np.einsum("bijc,bijo->co", xp[:, dy:dy + H, dx:dx + Wd], d)
            dxp[:, dy:dy + H, dx:dx + Wd] += np.einsum("bijo,co->bijc", d, Wt[dy, dx])
    return dxp[:, 1:-1, 1:-1], dW.reshape(W.shape), d.sum(axis=(0, 1, 2))


def forward(params, z, base, n_stages):
    """Output y [B, S, S, C_out] and the cache for backward."""
    z = np.asarray(z, dtype=np.float64)
    h1 = np.tanh(z @ params["W1"] + params["b1"])
    a2 = np.tanh(h1 @ params["W2"] + params["b2"])
    B = z.shape[0]
    x = a2.reshape(B, base, base, -1)
    cache = {"z": z, "h1": h1, "xs": [], "ups": [], "ys": []}
    for s, (wn, bn) in enumerate(stage_names(n_stages)):
        last = s == n_stages - 1
        u = x if last else up2(x)
        y = conv3x3(u, params[wn], params[bn])
        if not last:
            y = np.tanh(y)
        cache["xs"].append(x)
        cache["ups"].append(u)
        cache["ys"].append(y)
        x = y
    return x, cache


def backward(params, cache, dy, n_stages):
    """Gradients of every parameter for the output gradient dy."""
    grads = {}
    d = np.asarray(dy, dtype=np.float64)
    for s in reversed(range(n_stages)):
        wn, bn = stage_names(n_stages)[s]
        last = s == n_stages - 1
        if not last:
            d = d * (1.0 - cache["ys"][s] ** 2)
        du, grads[wn], grads[bn] = conv3x3_backward(cache["ups"][s], params[wn], d)
        d = du if last else up2_adjoint(du)
    B = d.shape[0]
    a2 = cache["xs"][0].reshape(B, -1)
    d2 = d.reshape(B, -1) * (1.0 - a2 ** 2)
    grads["W2"] = cache["h1"].T @ d2
    grads["b2"] = d2.sum(axis=0)
    dh1 = (d2 @ params["W2"].T) * (1.0 - cache["h1"] ** 2)
    grads["W1"] = cache["z"].T @ dh1
    grads["b1"] = dh1.sum(axis=0)
    return grads


def mse(y, t, wc=None):
    """Weighted mean squared error and its gradient with respect to y."""
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    w = np.ones(y.shape[-1]) if wc is None else np.asarray(wc, dtype=np.float64)
    n = y.size
    r = y - t
    return float((w * r * r).sum() / n), 2.0 * w * r / n


def adam(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (w, m, v) as new arrays."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    w = w - lr * (m / (1.0 - b1 ** t)) / (np.sqrt(v / (1.0 - b2 ** t)) + eps)
    return w, m, v

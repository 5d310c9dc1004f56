"""Warm-start network: predicts the steady cavity state from (log Ra, Pr, a).

Not part of the paper's method.  A small decoder network maps three scalars
to the temperature and velocity fields of the steady 2-D cavity on the mesh
index grid; islbm_set_fields_device then starts the solver from its
prediction (equilibrium initialisation) instead of from rest.

Architecture (about 1.1M parameters at the default size):
    z = features(log10 Ra, Pr, a), padded to 16
    h1 = tanh(z W1 + b1)                         256
    h2 = tanh(h1 W2 + b2)                        base x base x C0 (NHWC)
    for each stage: up 2x, 3x3 conv, tanh       channels C1 .. Cs
    y = 3x3 conv (no activation)                 3 channels: T* - 1/2, s u*, s v*

Every operation runs in the library's CUDA kernels (islbm_cnn_*): BF16
tensor-core GEMMs with FP32 accumulation for the fully connected layers and
the im2col convolutions, and elementwise kernels.  torch supplies device
memory and the stream only.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from .islbm import IslbmError, load_library

FEATURES = 16          # input features, padded for the tensor-core k-step
VEL_SCALE = 4.0        # u*, v* are learned as VEL_SCALE u*


def features(log10_ra, pr, a):
    """Normalised inputs (log Ra over [6, 8], Pr around 0.71, a around 1.5)."""
    z = np.zeros((len(log10_ra), FEATURES), dtype=np.float32)
    z[:, 0] = (np.asarray(log10_ra) - 7.0)
    z[:, 1] = (np.asarray(pr) - 0.71) * 2.0
    z[:, 2] = (np.asarray(a) - 1.5) * 2.0
    return z


def _ck(st):
    if st != 0:
        raise IslbmError(st, "warm-start network kernel")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class WarmStartNet:
    """The network, its parameters (FP32 masters + BF16 copies) and Adam state."""

    def __init__(self, base=8, channels=(64, 64, 48, 32, 16, 16), hidden=256, out_ch=3, seed=0,
                 device="cuda"):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.base, self.channels, self.hidden, self.out_ch = base, tuple(channels), hidden, out_ch
        self.size = base * 2 ** (len(channels) - 1)
        self.device = device
        g = np.random.default_rng(seed)
        shapes = [("W1", (FEATURES, hidden)), ("b1", (hidden,)),
                  ("W2", (hidden, base * base * channels[0])), ("b2", (base * base * channels[0],))]
        cin = channels[0]
        self.kpads = []
        for s, cout in enumerate(list(channels[1:]) + [out_ch]):
            kp = self._kpad(cin)
            self.kpads.append(kp)
            shapes += [(f"Wc{s}", (kp, cout)), (f"bc{s}", (cout,))]
            cin = cout
        self.names = [n for n, _ in shapes]
        self.params, self.bf, self.grads, self.m, self.v = {}, {}, {}, {}, {}
        for name, shp in shapes:
            if name.startswith("b"):
                w = np.zeros(shp, dtype=np.float32)
            else:
                fan_in = shp[0] if not name.startswith("Wc") else 9 * self._cin_of(name)
                w = (g.standard_normal(shp) * math.sqrt(1.0 / fan_in)).astype(np.float32)
                if name.startswith("Wc"):
                    w[9 * self._cin_of(name):] = 0.0         # padded rows stay zero
            self.params[name] = torch.from_numpy(w).to(device)
            self.grads[name] = torch.zeros_like(self.params[name])
            self.m[name] = torch.zeros_like(self.params[name])
            self.v[name] = torch.zeros_like(self.params[name])
            if name.startswith("W"):
                self.bf[name] = torch.empty(shp, dtype=torch.bfloat16, device=device)
                self._to_bf16(self.params[name], self.bf[name])
        self.t = 0
        self.n_params = int(sum(int(np.prod(s)) for n, s in shapes
                                if not n.startswith("Wc")) +
                            sum(9 * self._cin_of(n) * s[1] for n, s in shapes if n.startswith("Wc")))

    # ---- helpers ----
    @staticmethod
    def _kpad(c):
        return (9 * c + 15) // 16 * 16

    def _cin_of(self, name):
        s = int(name[2:])
        return self.channels[s]

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _to_bf16(self, x, y):
        _ck(self.lib.islbm_cnn_to_bf16(_p(x), _p(y), x.numel(), self._stream()))

    def _gemm(self, A, B, C, M, N, K, lda, ldb, ldc, ta=0, tb=0, bias=None, acc=0):
        _ck(self.lib.islbm_cnn_gemm_bf16(_p(A), _p(B), _p(C), _p(bias), M, N, K, lda, ldb, ldc,
                                         ta, tb, acc, self._stream()))

    # ---- forward ----
    def forward(self, z: np.ndarray, keep=True):
        """z: [B, 16] features.  Returns the output [B, S, S, 3] (torch, FP32)."""
        torch = self.torch
        B = z.shape[0]
        st = self._stream()
        cache = {"B": B}
        zt = torch.from_numpy(np.ascontiguousarray(z, dtype=np.float32)).to(self.device)
        zb = torch.empty_like(zt, dtype=torch.bfloat16)
        self._to_bf16(zt, zb)
        h1 = torch.empty((B, self.hidden), device=self.device)
        self._gemm(zb, self.bf["W1"], h1, B, self.hidden, FEATURES, FEATURES, self.hidden,
                   self.hidden, bias=self.params["b1"])
        _ck(self.lib.islbm_cnn_tanh(_p(h1), h1.numel(), st))
        h1b = torch.empty_like(h1, dtype=torch.bfloat16)
        self._to_bf16(h1, h1b)
        n2 = self.base * self.base * self.channels[0]
        x = torch.empty((B, self.base, self.base, self.channels[0]), device=self.device)
        self._gemm(h1b, self.bf["W2"], x, B, n2, self.hidden, self.hidden, n2, n2,
                   bias=self.params["b2"])
        _ck(self.lib.islbm_cnn_tanh(_p(x), x.numel(), st))
        cache.update(zb=zb, h1=h1, h1b=h1b, stages=[])
        H = self.base
        cin = self.channels[0]
        outs = list(self.channels[1:]) + [self.out_ch]
        for s, cout in enumerate(outs):
            last = s == len(outs) - 1
            if not last:
                up = torch.empty((B, 2 * H, 2 * H, cin), device=self.device)
                _ck(self.lib.islbm_cnn_upsample2x(_p(x), _p(up), B, H, H, cin, 0, st))
                H *= 2
            else:
                up = x
            kp = self.kpads[s]
            col = torch.empty((B * H * H, kp), dtype=torch.bfloat16, device=self.device)
            _ck(self.lib.islbm_cnn_im2col(_p(up), _p(col), B, H, H, cin, kp, st))
            y = torch.empty((B, H, H, cout), device=self.device)
            self._gemm(col, self.bf[f"Wc{s}"], y, B * H * H, cout, kp, kp, cout, cout,
                       bias=self.params[f"bc{s}"])
            if not last:
                _ck(self.lib.islbm_cnn_tanh(_p(y), y.numel(), st))
            cache["stages"].append(dict(x=x, up=up, col=col, y=y, H=H, cin=cin, cout=cout,
                                        upsampled=not last))
            x, cin = y, cout
        self.cache = cache if keep else None
        return x

    # ---- backward ----
    def backward(self, dy):
        """Gradients of all parameters for the output gradient dy [B, S, S, 3]."""
        torch = self.torch
        c = self.cache
        B = c["B"]
        st = self._stream()
        d = dy.contiguous()
        for s in reversed(range(len(c["stages"]))):
            g = c["stages"][s]
            H, cin, cout, kp = g["H"], g["cin"], g["cout"], self.kpads[s]
            last = s == len(c["stages"]) - 1
            if not last:
                _ck(self.lib.islbm_cnn_tanh_back(_p(g["y"]), _p(d), d.numel(), st))
            M = B * H * H
            db = torch.empty((M, cout), dtype=torch.bfloat16, device=self.device)
            self._to_bf16(d, db)
            # dW = col^T dY, db = colsum(dY)
            self._gemm(g["col"], db, self.grads[f"Wc{s}"], kp, cout, M, kp, cout, cout, ta=1)
            _ck(self.lib.islbm_cnn_colsum(_p(d), _p(self.grads[f"bc{s}"]), M, cout, 0, st))
            # dcol = dY W^T, dup = col2im(dcol), dx = up^T(dup)
            dcol = torch.empty((M, kp), device=self.device)
            self._gemm(db, self.bf[f"Wc{s}"], dcol, M, kp, cout, cout, cout, kp, tb=1)
            dup = torch.empty((B, H, H, cin), device=self.device)
            _ck(self.lib.islbm_cnn_col2im(_p(dcol), _p(dup), B, H, H, cin, kp, st))
            if g["upsampled"]:
                dx = torch.empty((B, H // 2, H // 2, cin), device=self.device)
                _ck(self.lib.islbm_cnn_upsample2x(_p(dup), _p(dx), B, H // 2, H // 2, cin, 1, st))
            else:
                dx = dup
            d = dx
        # fully connected layers
        n2 = self.base * self.base * self.channels[0]
        x0 = c["stages"][0]["x"]
        _ck(self.lib.islbm_cnn_tanh_back(_p(x0), _p(d), d.numel(), st))
        d2 = d.reshape(B, n2)
        d2b = torch.empty_like(d2, dtype=torch.bfloat16)
        self._to_bf16(d2, d2b)
        self._gemm(c["h1b"], d2b, self.grads["W2"], self.hidden, n2, B, self.hidden, n2, n2, ta=1)
        _ck(self.lib.islbm_cnn_colsum(_p(d2), _p(self.grads["b2"]), B, n2, 0, st))
        dh1 = torch.empty((B, self.hidden), device=self.device)
        self._gemm(d2b, self.bf["W2"], dh1, B, self.hidden, n2, n2, n2, self.hidden, tb=1)
        _ck(self.lib.islbm_cnn_tanh_back(_p(c["h1"]), _p(dh1), dh1.numel(), st))
        dh1b = torch.empty_like(dh1, dtype=torch.bfloat16)
        self._to_bf16(dh1, dh1b)
        self._gemm(c["zb"], dh1b, self.grads["W1"], FEATURES, self.hidden, B, FEATURES,
                   self.hidden, self.hidden, ta=1)
        _ck(self.lib.islbm_cnn_colsum(_p(dh1), _p(self.grads["b1"]), B, self.hidden, 0, st))
        return self.grads

    def mse(self, y, target, weights=None):
        """Mean squared error and its gradient (islbm_cnn_mse)."""
        torch = self.torch
        n = y.numel()
        blocks = 256
        dy = torch.empty_like(y)
        part = torch.empty(blocks, dtype=torch.float64, device=self.device)
        _ck(self.lib.islbm_cnn_mse(_p(y), _p(target), _p(weights), self.out_ch, _p(dy), _p(part),
                                   blocks, n, self._stream()))
        return part, dy

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        st = self._stream()
        for name in self.names:
            w = self.params[name]
            _ck(self.lib.islbm_cnn_adam(_p(w), _p(self.bf.get(name)), _p(self.grads[name]),
                                        _p(self.m[name]), _p(self.v[name]), w.numel(),
                                        ctypes.c_float(lr), ctypes.c_float(b1), ctypes.c_float(b2),
                                        ctypes.c_float(eps), self.t, st))

    # ---- parameters to / from numpy (checkpoints, oracle comparisons) ----
    def numpy_params(self):
        out = {}
        for name in self.names:
            w = self.params[name].detach().cpu().numpy()
            if name.startswith("Wc"):
                w = w[:9 * self._cin_of(name)]
            out[name] = w
        return out

    def load_numpy_params(self, params):
        for name in self.names:
            w = np.array(params[name], dtype=np.float32)
            if name.startswith("Wc"):
                full = np.zeros(self.params[name].shape, dtype=np.float32)
                full[:w.shape[0]] = w
                w = full
            self.params[name].copy_(self.torch.from_numpy(w))
            if name in self.bf:
                self._to_bf16(self.params[name], self.bf[name])

    def predict_fields(self, log10_ra, pr, a):
        """Predicted T (in wall units, walls +-1/2), u*, v* on the S x S grid per input."""
        y = self.forward(features(log10_ra, pr, a), keep=False)
        out = y.detach().cpu().numpy().astype(np.float64)
        return out[..., 0], out[..., 1] / VEL_SCALE, out[..., 2] / VEL_SCALE

"""GPU parity of the warm-start network's kernels against the float64 oracle.

Tolerances.  The GEMM kernel multiplies BF16 operands exactly and accumulates
in FP32, so against the float64 product of the same BF16-rounded operands its
error is FP32 accumulation only: with random signs about sqrt(L) 2^-24 of
sum |a||b| for a summation length L (at most a few hundred per accumulator,
the split-K parts included), checked at 1e-5 of that scale.  The whole
network rounds every GEMM operand to BF16 (unit roundoff 2^-9); five layers
of such products with contractive tanh activations give a relative error of
about sqrt(5) x 2 x 2^-9 ~ 1e-2 in the output, and the backward pass rounds
its incoming gradients once more, so outputs are checked at 2e-2 and
gradients at 4e-2 in relative Frobenius norm.
"""
import ctypes

import numpy as np
import pytest

from oracle import cnn_oracle as oc
from synthetic import gaussian_arrays
from tests.helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA device")]


def _torch():
    import torch
    return torch


def _lib():
    from paper_2509_01099_gb300.islbm import load_library
    return load_library()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _bf16_round(x):
    torch = _torch()
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("M,N,K,ta,tb", [
    (70, 45, 37, 0, 0), (130, 64, 96, 1, 0), (33, 150, 48, 0, 1), (65, 66, 70, 1, 1),
    (144, 16, 40000, 1, 0),     # the weight-gradient shape: split over K
    (5, 4096, 256, 0, 0),       # the second fully connected layer
])
def test_gemm_bf16_matches_float64_of_rounded_operands(M, N, K, ta, tb):
    torch = _torch()
    g = gaussian_arrays([("A", (K, M) if ta else (M, K)), ("B", (N, K) if tb else (K, N)),
                         ("bias", (N,)), ("C0", (M, N))], seed=M + N + K)
    A = torch.from_numpy(g["A"].astype(np.float32)).cuda().to(torch.bfloat16)
    B = torch.from_numpy(g["B"].astype(np.float32)).cuda().to(torch.bfloat16)
    bias = torch.from_numpy(g["bias"].astype(np.float32)).cuda()
    C = torch.from_numpy(g["C0"].astype(np.float32)).cuda()
    lda, ldb = A.shape[1], B.shape[1]
    lib = _lib()
    for acc in (0, 1):
        Cin = C.clone()
        st = lib.islbm_cnn_gemm_bf16(_p(A), _p(B), _p(Cin), _p(bias), M, N, K, lda, ldb, N,
                                     ta, tb, acc, _stream())
        assert st == 0
        torch.cuda.synchronize()
        Ar, Br = _bf16_round(g["A"]), _bf16_round(g["B"])
        opA = Ar.T if ta else Ar
        opB = Br.T if tb else Br
        ref = opA @ opB + g["bias"].astype(np.float32)
        if acc:
            ref = ref + g["C0"].astype(np.float32)
        scale = np.abs(opA) @ np.abs(opB) + np.abs(g["bias"]) + (np.abs(g["C0"]) if acc else 0)
        err = np.abs(Cin.cpu().numpy() - ref) / scale
        assert err.max() < 1e-5, err.max()


def _gemm_case(M, N, K, ta, tb, seed, path, acc=0, lda_pad=0, ldb_pad=0):
    """One product through islbm_cnn_gemm_bf16_ex; returns (C, reference, scale)."""
    torch = _torch()
    ashape = (K, M + lda_pad) if ta else (M, K + lda_pad)
    bshape = (N, K + ldb_pad) if tb else (K, N + ldb_pad)
    g = gaussian_arrays([("A", ashape), ("B", bshape), ("bias", (N,)), ("C0", (M, N))],
                        seed=seed)
    A = torch.from_numpy(g["A"].astype(np.float32)).cuda().to(torch.bfloat16)
    B = torch.from_numpy(g["B"].astype(np.float32)).cuda().to(torch.bfloat16)
    bias = torch.from_numpy(g["bias"].astype(np.float32)).cuda()
    C = torch.from_numpy(g["C0"].astype(np.float32)).cuda()
    lda, ldb = A.shape[1], B.shape[1]
    st = _lib().islbm_cnn_gemm_bf16_ex(_p(A), _p(B), _p(C), _p(bias), M, N, K, lda, ldb, N,
                                       ta, tb, acc, path, _stream())
    assert st == 0
    torch.cuda.synchronize()
    Ar, Br = _bf16_round(g["A"]), _bf16_round(g["B"])
    opA = Ar[:, :M].T if ta else Ar[:, :K]
    opB = Br[:, :K].T if tb else Br[:, :N]
    ref = opA @ opB + g["bias"].astype(np.float32) + (g["C0"].astype(np.float32) if acc else 0)
    scale = np.abs(opA) @ np.abs(opB) + np.abs(g["bias"]) + (np.abs(g["C0"]) if acc else 0)
    return C.cpu().numpy(), ref, scale


# Shapes of the tcgen05 path: every N tile width (16 .. 256, ragged N), ragged M
# and K ends (a k stage cut inside its 64 values, K below one stage), all four
# operand orientations, the network's own products (forward im2col x W, data
# gradient dY x W^T, weight gradient col^T x dY over 256^2 x 16 nodes), padded
# leading dimensions, bias and accumulation.
TC_CASES = [
    (128, 16, 64, 0, 0), (200, 3, 40, 0, 1), (256, 32, 576, 0, 0), (300, 48, 432, 0, 0),
    (1000, 64, 144, 0, 0), (129, 100, 70, 1, 0), (96, 128, 24, 0, 1), (64, 200, 200, 1, 1),
    (517, 256, 136, 0, 1), (130, 600, 96, 0, 1),
    (65536, 16, 144, 0, 0),        # forward of the last 3x3 stage at 256^2 (one sample)
    (16384, 576, 64, 0, 1),        # data gradient dY W^T of a 64-channel stage
    (576, 64, 65536, 1, 0),        # weight gradient col^T dY: split over K
    (16, 4096, 256, 0, 0),         # the second fully connected layer (16 samples)
]


@pytest.mark.parametrize("M,N,K,ta,tb", TC_CASES)
def test_gemm_tcgen05_matches_float64_of_rounded_operands(M, N, K, ta, tb):
    # leading dimensions rounded up to 8 elements (the path's condition), then
    # a further padding of one and two chunks
    la, lb = (M if ta else K), (K if tb else N)
    base = ((-la) % 8, (-lb) % 8)
    for acc, extra in ((0, (0, 0)), (1, (8, 16))):
        C, ref, scale = _gemm_case(M, N, K, ta, tb, seed=M + 3 * N + 7 * K + ta + 2 * tb,
                                   path=2, acc=acc, lda_pad=base[0] + extra[0],
                                   ldb_pad=base[1] + extra[1])
        err = np.abs(C - ref) / scale
        assert err.max() < 1e-5, (acc, err.max())
    flag = ctypes.c_int(-1)
    assert _lib().islbm_cnn_check_timeout(1, ctypes.byref(flag)) == 0 and flag.value == 0


def test_gemm_split_k_is_deterministic_on_both_paths():
    """The weight-gradient shape (split over K): two runs of either path give
    the same bits (the splits are added in a fixed order); the paths agree
    within the accumulation tolerance."""
    a, ref, scale = _gemm_case(576, 64, 65536, 1, 0, seed=5, path=2)
    b, _, _ = _gemm_case(576, 64, 65536, 1, 0, seed=5, path=2)
    c, _, _ = _gemm_case(576, 64, 65536, 1, 0, seed=5, path=1)
    d, _, _ = _gemm_case(576, 64, 65536, 1, 0, seed=5, path=1)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(c, d)
    assert (np.abs(a - c) / scale).max() < 2e-5


def test_gemm_tcgen05_refuses_unaligned_operands():
    torch = _torch()
    lib = _lib()
    A = torch.zeros(4096, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(4096, device="cuda")
    # lda = 37 is not a multiple of 8 elements: path 2 refuses, path 0 takes mma.sync
    assert lib.islbm_cnn_gemm_bf16_ex(_p(A), _p(A), _p(C), None, 8, 8, 37, 37, 8, 8, 0, 0, 0, 2,
                                      _stream()) != 0
    assert lib.islbm_cnn_gemm_bf16_ex(_p(A), _p(A), _p(C), None, 8, 8, 37, 37, 8, 8, 0, 0, 0, 0,
                                      _stream()) == 0
    torch.cuda.synchronize()


def test_gemm_rejects_bad_sizes():
    torch = _torch()
    lib = _lib()
    A = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, device="cuda")
    assert lib.islbm_cnn_gemm_bf16(_p(A), _p(A), _p(C), None, 0, 8, 8, 8, 8, 8, 0, 0, 0,
                                   _stream()) != 0
    assert lib.islbm_cnn_gemm_bf16(_p(A), _p(A), _p(C), None, 8, 8, 8, 4, 8, 8, 0, 0, 0,
                                   _stream()) != 0    # lda < K


def test_im2col_col2im_upsample_colsum():
    torch = _torch()
    lib = _lib()
    B, H, W, C, kp = 2, 9, 7, 5, 48
    g = gaussian_arrays([("x", (B, H, W, C)), ("d", (B * H * W, kp)), ("u", (B, 2 * H, 2 * W, C))],
                        seed=11)
    x = torch.from_numpy(g["x"].astype(np.float32)).cuda()
    col = torch.empty((B * H * W, kp), dtype=torch.bfloat16, device="cuda")
    assert lib.islbm_cnn_im2col(_p(x), _p(col), B, H, W, C, kp, _stream()) == 0
    # im2col of x times a one-hot kernel is the conv of the oracle with that kernel
    xr = _bf16_round(g["x"])
    got = col.to(torch.float64).cpu().numpy()
    for tap in range(9):
        Wk = np.zeros((9 * C, C))
        Wk[tap * C:(tap + 1) * C] = np.eye(C)
        ref = oc.conv3x3(xr, Wk, np.zeros(C)).reshape(-1, C)
        assert np.array_equal(got[:, tap * C:(tap + 1) * C], ref)
    assert not got[:, 9 * C:].any()
    # col2im is the adjoint: <im2col(x), d> = <x, col2im(d)> with d zero in the pad
    d = g["d"].copy()
    d[:, 9 * C:] = 0.0
    dd = torch.from_numpy(d.astype(np.float32)).cuda()
    din = torch.empty_like(x)
    assert lib.islbm_cnn_col2im(_p(dd), _p(din), B, H, W, C, kp, _stream()) == 0
    lhs = np.vdot(got, d.astype(np.float32))
    rhs = np.vdot(xr, din.cpu().numpy().astype(np.float64))
    assert abs(lhs - rhs) < 1e-5 * np.abs(got).sum() * np.abs(d).max()
    # upsampling and its adjoint
    up = torch.empty((B, 2 * H, 2 * W, C), device="cuda")
    assert lib.islbm_cnn_upsample2x(_p(x), _p(up), B, H, W, C, 0, _stream()) == 0
    assert np.array_equal(up.cpu().numpy(), oc.up2(g["x"].astype(np.float32)))
    u = torch.from_numpy(g["u"].astype(np.float32)).cuda()
    back = torch.empty_like(x)
    assert lib.islbm_cnn_upsample2x(_p(u), _p(back), B, H, W, C, 1, _stream()) == 0
    np.testing.assert_allclose(back.cpu().numpy(), oc.up2_adjoint(g["u"]), rtol=0, atol=2e-6)
    # column sums over many row chunks
    big = gaussian_arrays([("m", (10000, 37))], seed=12)["m"]
    bt = torch.from_numpy(big.astype(np.float32)).cuda()
    out = torch.full((37,), 5.0, device="cuda")
    assert lib.islbm_cnn_colsum(_p(bt), _p(out), 10000, 37, 0, _stream()) == 0
    np.testing.assert_allclose(out.cpu().numpy(), big.sum(axis=0), rtol=0, atol=2e-3)
    first = out.cpu().numpy().copy()
    assert lib.islbm_cnn_colsum(_p(bt), _p(out), 10000, 37, 1, _stream()) == 0
    np.testing.assert_allclose(out.cpu().numpy(), 2 * big.sum(axis=0), rtol=0, atol=4e-3)
    # the row chunks are added in a fixed order: a repeat gives the same bits
    assert lib.islbm_cnn_colsum(_p(bt), _p(out), 10000, 37, 0, _stream()) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), first)


def test_mse_tanh_adam_against_oracle():
    torch = _torch()
    lib = _lib()
    g = gaussian_arrays([("y", (3, 8, 8, 3)), ("t", (3, 8, 8, 3)), ("w", (500,)),
                         ("g1", (500,)), ("g2", (500,)), ("g3", (500,))], seed=13)
    y = torch.from_numpy(g["y"].astype(np.float32)).cuda()
    t = torch.from_numpy(g["t"].astype(np.float32)).cuda()
    wc = torch.tensor([1.0, 0.5, 2.0], device="cuda")
    dy = torch.empty_like(y)
    part = torch.empty(64, dtype=torch.float64, device="cuda")
    assert lib.islbm_cnn_mse(_p(y), _p(t), _p(wc), 3, _p(dy), _p(part), 64, y.numel(),
                             _stream()) == 0
    loss_ref, dy_ref = oc.mse(g["y"].astype(np.float32), g["t"].astype(np.float32), [1.0, 0.5, 2.0])
    assert abs(part.sum().item() / y.numel() - loss_ref) < 1e-6 * loss_ref
    np.testing.assert_allclose(dy.cpu().numpy(), dy_ref, rtol=1e-6, atol=1e-12)
    # tanh and its derivative
    x = y.clone()
    assert lib.islbm_cnn_tanh(_p(x), x.numel(), _stream()) == 0
    np.testing.assert_allclose(x.cpu().numpy(), np.tanh(g["y"]), rtol=0, atol=2e-6)
    d = t.clone()
    assert lib.islbm_cnn_tanh_back(_p(x), _p(d), d.numel(), _stream()) == 0
    th = x.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(d.cpu().numpy(), g["t"] * (1 - th ** 2), rtol=1e-6, atol=1e-7)
    # three Adam steps with changing gradients
    w = torch.from_numpy(g["w"].astype(np.float32)).cuda()
    wb = torch.empty(500, dtype=torch.bfloat16, device="cuda")
    m = torch.zeros(500, device="cuda")
    v = torch.zeros(500, device="cuda")
    wr, mr, vr = g["w"].astype(np.float32).astype(np.float64), np.zeros(500), np.zeros(500)
    for step, gn in enumerate(("g1", "g2", "g3"), start=1):
        gg = torch.from_numpy(g[gn].astype(np.float32)).cuda()
        assert lib.islbm_cnn_adam(_p(w), _p(wb), _p(gg), _p(m), _p(v), 500, ctypes.c_float(1e-2),
                                  ctypes.c_float(0.9), ctypes.c_float(0.999),
                                  ctypes.c_float(1e-8), step, _stream()) == 0
        wr, mr, vr = oc.adam(wr, g[gn].astype(np.float32), mr, vr, step, lr=1e-2)
    np.testing.assert_allclose(w.cpu().numpy(), wr, rtol=0, atol=2e-6)
    assert np.array_equal(wb.to(torch.float32).cpu().numpy(),
                          w.to(torch.bfloat16).to(torch.float32).cpu().numpy())


def _small_net(seed):
    from paper_2509_01099_gb300.cnn import WarmStartNet, FEATURES
    net = WarmStartNet(base=4, channels=(32, 24, 16), hidden=64, out_ch=3, seed=seed)
    shapes = [("W1", (FEATURES, 64)), ("b1", (64,)), ("W2", (64, 4 * 4 * 32)),
              ("b2", (4 * 4 * 32,))]
    cin = 32
    for s, cout in enumerate([24, 16, 3]):
        shapes += [(f"Wc{s}", (9 * cin, cout)), (f"bc{s}", (cout,))]
        cin = cout
    scales = {n: (1.0 / np.sqrt(9 * net._cin_of(n)) if n.startswith("Wc") else
                  1.0 / np.sqrt(shp[0]) if n.startswith("W") else 0.1) for n, shp in shapes}
    params = gaussian_arrays(shapes, seed, scales)
    net.load_numpy_params(params)
    # the oracle takes the weights as the network holds them (FP32 masters)
    return net, {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}


def test_network_forward_backward_matches_oracle():
    torch = _torch()
    net, params = _small_net(seed=21)
    g = gaussian_arrays([("z", (5, 16)), ("t", (5, 16, 16, 3))], seed=22)
    y = net.forward(g["z"].astype(np.float32))
    yo, cache = oc.forward(params, g["z"].astype(np.float32), 4, 3)
    assert y.shape == (5, 16, 16, 3)
    assert _rel(y.cpu().numpy(), yo) < 2e-2
    tgt = torch.from_numpy(g["t"].astype(np.float32)).cuda()
    wc = torch.tensor([2.0, 1.0, 1.0], device="cuda")
    part, dy = net.mse(y, tgt, wc)
    loss_o, dy_o = oc.mse(yo, g["t"].astype(np.float32), [2.0, 1.0, 1.0])
    assert abs(part.sum().item() / y.numel() - loss_o) < 2e-2 * loss_o
    grads = net.backward(dy)
    go = oc.backward(params, cache, dy_o, 3)
    for name in net.names:
        gg = grads[name].cpu().numpy().astype(np.float64)
        if name.startswith("Wc"):
            assert not gg[9 * net._cin_of(name):].any()     # padded rows get no gradient
            gg = gg[:9 * net._cin_of(name)]
        assert _rel(gg, go[name]) < 4e-2, (name, _rel(gg, go[name]))


def test_training_lowers_the_loss():
    torch = _torch()
    net, _ = _small_net(seed=31)
    g = gaussian_arrays([("z", (8, 16))], seed=32)
    # a smooth target that depends on the input: the network must fit it
    yy, xx = np.meshgrid(np.linspace(-1, 1, 16), np.linspace(-1, 1, 16), indexing="ij")
    t = np.stack([np.tanh(g["z"][:, :1, None] * xx[None] + yy[None] * 0.5),
                  0.3 * np.sin(np.pi * xx)[None].repeat(8, 0),
                  g["z"][:, 1:2, None] * yy[None] * 0.2], axis=-1).astype(np.float32)
    tgt = torch.from_numpy(t).cuda()
    losses = []
    for _ in range(200):
        y = net.forward(g["z"].astype(np.float32))
        part, dy = net.mse(y, tgt)
        losses.append(part.sum().item() / y.numel())
        net.backward(dy)
        net.adam(lr=3e-3)
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def test_pack_and_unpack_fields():
    """Solver fields <-> network channels: pack divides by the scales in FP64
    and rounds once to FP32; unpack is its inverse to that rounding."""
    torch = _torch()
    lib = _lib()
    g = gaussian_arrays([("T", (300,)), ("u", (300,)), ("v", (300,))], seed=51)
    T = torch.from_numpy(0.4 * g["T"]).cuda()
    u = torch.from_numpy(0.01 * g["u"]).cuda()
    v = torch.from_numpy(0.01 * g["v"]).cuda()
    y = torch.empty((300, 3), device="cuda")
    T_mid, T_scale, u_scale = 0.1, 2.0, 0.0125
    assert lib.islbm_cnn_pack_fields(_p(T), _p(u), _p(v), 300, ctypes.c_double(T_mid),
                                     ctypes.c_double(T_scale), ctypes.c_double(u_scale), _p(y),
                                     _stream()) == 0
    yy = y.cpu().numpy()
    np.testing.assert_array_equal(yy[:, 0], ((0.4 * g["T"] - T_mid) / T_scale).astype(np.float32))
    np.testing.assert_array_equal(yy[:, 1], (0.01 * g["u"] / u_scale).astype(np.float32))
    T2, u2, v2 = torch.empty_like(T), torch.empty_like(u), torch.empty_like(v)
    assert lib.islbm_cnn_unpack_fields(_p(y), 300, ctypes.c_double(T_mid),
                                       ctypes.c_double(T_scale), ctypes.c_double(u_scale),
                                       _p(T2), _p(u2), _p(v2), _stream()) == 0
    for a, b in ((T2, T), (u2, u), (v2, v)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(a - b).max() <= 2 ** -23 * np.abs(b).max() * 4
    # a zero scale is rejected
    assert lib.islbm_cnn_pack_fields(_p(T), _p(u), _p(v), 300, ctypes.c_double(0.0),
                                     ctypes.c_double(0.0), ctypes.c_double(1.0), _p(y),
                                     _stream()) != 0

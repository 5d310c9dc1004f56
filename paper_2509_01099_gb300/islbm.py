"""ctypes binding of libislbm (include/islbm.h).

The functions below carry the names of the C entry points and only marshal
arguments: numpy arrays for host buffers, torch CUDA tensors (or raw device
addresses) for device buffers, and torch's current CUDA stream by default.
Every computation runs in the library's CUDA kernels; there is no CPU path.
If the library has not been built the first call raises ``IslbmError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LATTICES = {"d2q9_d2q5": 0, "d3q19_d3q7": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16dev": 2, "bf16dev": 3, "fp16neq": 4}
STENCILS = {"centred": 0, "upwind": 1}
REFERENCES = {"mean": 0, "cold": 1}
KERNEL_VARIANTS = 10     # ISLBM_KERNEL_VARIANTS of include/islbm.h
KERNELS = {"auto": 0, "direct": 1, "tiled": 2, "tma_r4s2": 3, "tma_r2s2": 4, "tma_r2s3": 5,
           "tma_r4s3": 6, "tma3d": 7, "zm3d": 8, "zm3d_t4": 9}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_DIVERGED",
          5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_IO"}

# symbols declared in include/islbm.h
EXPORTS = (
    "islbm_mesh_uniform", "islbm_mesh_erf", "islbm_mesh_tanh", "islbm_default_params",
    "islbm_create", "islbm_destroy", "islbm_last_error", "islbm_info",
    "islbm_set_fields", "islbm_set_fields_device", "islbm_set_populations", "islbm_step",
    "islbm_get_fields", "islbm_get_fields_device", "islbm_get_populations", "islbm_reduce",
    "islbm_nusselt", "islbm_reynolds", "islbm_mass", "islbm_synchronize", "islbm_save",
    "islbm_load", "islbm_reduce_noalloc", "islbm_steady_change", "islbm_run_to_steady",
    "islbm_autotune", "islbm_batch_create", "islbm_batch_destroy", "islbm_batch_member",
    "islbm_batch_tile_rows", "islbm_batch_step", "islbm_batch_synchronize",
    "islbm_batch_run_to_steady", "islbm_batch_run_to_steady_nu", "islbm_average_reset",
    "islbm_average_add", "islbm_average_get", "islbm_debug_bounds", "islbm_selftest_wait_timeout",
    "islbm_selftest_wait_abort",
    "islbm_cnn_gemm_bf16", "islbm_cnn_im2col", "islbm_cnn_col2im",
    "islbm_cnn_upsample2x", "islbm_cnn_tanh", "islbm_cnn_tanh_back", "islbm_cnn_to_bf16",
    "islbm_cnn_colsum", "islbm_cnn_mse", "islbm_cnn_adam", "islbm_cnn_pack_fields",
    "islbm_cnn_unpack_fields", "islbm_set_row_range", "islbm_get_rows", "islbm_set_rows",
    "islbm_reduce_sums", "islbm_finish_sums", "islbm_cnn_gemm_bf16_ex", "islbm_cnn_check_timeout",
    "islbm_set_allocator",
)
REDUCTION_SUMS = 16     # ISLBM_REDUCTION_SUMS of include/islbm.h
SUM_MAX_SLOT = 13       # ISLBM_SUM_MAX_SLOT: the one partial combined by max
MESH_KINDS = {"uniform": 0, "erf": 1, "tanh": 2}


class IslbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"islbm {STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("Ma", ctypes.c_double), ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double),
                ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
                ("s_pi", ctypes.c_double), ("s_m", ctypes.c_double), ("q_j", ctypes.c_double),
                ("q_e", ctypes.c_double), ("q_nu", ctypes.c_double), ("stencil", ctypes.c_int),
                ("kernel", ctypes.c_int), ("reference", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("q_flow", ctypes.c_int),
                ("q_temp", ctypes.c_int), ("uniform", ctypes.c_int), ("precision", ctypes.c_int),
                ("L", ctypes.c_double), ("u_f", ctypes.c_double), ("nu", ctypes.c_double),
                ("alpha", ctypes.c_double), ("gbeta", ctypes.c_double), ("s_nu", ctypes.c_double),
                ("a_T", ctypes.c_double), ("omega", ctypes.c_double),
                ("steps_per_tf", ctypes.c_double), ("bytes_per_update", ctypes.c_double),
                ("time", ctypes.c_longlong), ("kernel", ctypes.c_int), ("sm_count", ctypes.c_int)]


class Reductions(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("Nu", "Nu_hot", "Nu_cold", "Nu_middle", "Re", "Re_uv", "Re_mean", "mass", "ke",
                 "max_speed", "nonfinite")] + [("time", ctypes.c_longlong)]


class Cavity(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("mesh", ctypes.c_int), ("a", ctypes.c_double),
                ("Ra", ctypes.c_double), ("Pr", ctypes.c_double)]


class NuOut(ctypes.Structure):
    _fields_ = [("vol", ctypes.c_double), ("hot", ctypes.c_double), ("cold", ctypes.c_double),
                ("middle", ctypes.c_double)]


_lib = None


def library_path() -> str:
    """The library to load: $ISLBM_LIBRARY if set (e.g. the bounds-checked
    build), else the in-tree libislbm.so."""
    return os.environ.get("ISLBM_LIBRARY") or _build.LIB


# device-memory callbacks of islbm_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
# Every callback ever registered stays referenced for the life of the process:
# handles (and the network's workspace) keep the allocator they were created
# with and call its release function when they are destroyed, possibly after
# another allocator has been registered.
_allocator_refs = []


def islbm_set_allocator(alloc=None, release=None):
    """Register Python callables alloc(nbytes, device, stream) -> int pointer and
    release(ptr, device, stream) as the library's device allocator (None, None:
    back to cudaMallocAsync on the owner's stream)."""
    lib = load_library()
    if alloc is None and release is None:
        _check(lib.islbm_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _a(nbytes, device, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(device), int(stream or 0))) or None
        except Exception:     # noqa: BLE001 - a NULL return is the library's OOM
            return None

    def _r(ptr, device, stream, ctx):
        try:
            release(int(ptr), int(device), int(stream or 0))
        except Exception:     # noqa: BLE001
            pass

    fa, fr = ALLOC_FN(_a), FREE_FN(_r)
    _allocator_refs.extend([fa, fr, _a, _r])
    _check(lib.islbm_set_allocator(fa, fr, None))


def torch_allocator():
    """(alloc, release) on torch's CUDA caching allocator."""
    import torch

    def alloc(nbytes, device, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device=device, stream=stream)

    def release(ptr, device, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, release


def load_library(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libislbm.so (optionally building it first).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise IslbmError(2, f"{path} is not built; run paper_2509_01099_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    d, i, vp, h = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    dp = P(ctypes.c_double)
    sig = {
        "islbm_mesh_uniform": (i, [i, dp]),
        "islbm_mesh_erf": (i, [i, d, dp]),
        "islbm_mesh_tanh": (i, [i, d, dp]),
        "islbm_default_params": (None, [P(Params)]),
        "islbm_create": (i, [dp, i, dp, i, dp, i, d, d, i, i, P(Params), vp, P(h)]),
        "islbm_destroy": (None, [h]),
        "islbm_last_error": (ctypes.c_char_p, [h]),
        "islbm_info": (i, [h, P(Info)]),
        "islbm_set_fields": (i, [h, dp, dp, dp, dp, dp]),
        "islbm_set_fields_device": (i, [h, vp, vp, vp, vp, vp]),
        "islbm_set_populations": (i, [h, dp, dp]),
        "islbm_step": (i, [h, ctypes.c_longlong]),
        "islbm_get_fields": (i, [h, dp, dp, dp, dp, dp]),
        "islbm_get_fields_device": (i, [h, vp, vp, vp, vp, vp]),
        "islbm_get_populations": (i, [h, dp, dp]),
        "islbm_reduce": (i, [h, P(Reductions)]),
        "islbm_nusselt": (i, [h, P(NuOut)]),
        "islbm_reynolds": (i, [h, dp]),
        "islbm_mass": (i, [h, dp]),
        "islbm_synchronize": (i, [h]),
        "islbm_save": (i, [h, ctypes.c_char_p]),
        "islbm_load": (i, [h, ctypes.c_char_p]),
        "islbm_reduce_noalloc": (i, [vp, vp, i, i, vp, vp, d, d, P(Params), vp, P(Reductions)]),
        "islbm_steady_change": (i, [h, dp, dp]),
        "islbm_autotune": (i, [i, i, d, i, vp, P(i), dp]),
        "islbm_batch_create": (i, [i, P(Cavity), i, P(Params), i, vp, P(h)]),
        "islbm_batch_destroy": (None, [h]),
        "islbm_batch_member": (i, [h, i, P(h)]),
        "islbm_batch_tile_rows": (i, [h, i]),
        "islbm_batch_step": (i, [h, ctypes.c_longlong]),
        "islbm_batch_synchronize": (i, [h]),
        "islbm_debug_bounds": (i, [i, P(i)]),
        "islbm_selftest_wait_timeout": (i, [vp]),
        "islbm_selftest_wait_abort": (i, [vp, P(ctypes.c_int), P(ctypes.c_int)]),
        "islbm_average_reset": (i, [h]),
        "islbm_average_add": (i, [h]),
        "islbm_average_get": (i, [h, dp, dp, dp, dp, P(ctypes.c_longlong)]),
        "islbm_batch_run_to_steady_nu": (i, [h, d, ctypes.c_longlong, i, ctypes.c_longlong,
                                             P(ctypes.c_longlong), dp, dp]),
        "islbm_batch_run_to_steady": (i, [h, d, ctypes.c_longlong, ctypes.c_longlong,
                                          P(ctypes.c_longlong)]),
        "islbm_cnn_gemm_bf16": (i, [vp, vp, vp, vp, i, i, i, i, i, i, i, i, i, vp]),
        "islbm_cnn_gemm_bf16_ex": (i, [vp, vp, vp, vp, i, i, i, i, i, i, i, i, i, i, vp]),
        "islbm_cnn_check_timeout": (i, [i, P(i)]),
        "islbm_cnn_im2col": (i, [vp, vp, i, i, i, i, i, vp]),
        "islbm_cnn_col2im": (i, [vp, vp, i, i, i, i, i, vp]),
        "islbm_cnn_upsample2x": (i, [vp, vp, i, i, i, i, i, vp]),
        "islbm_cnn_tanh": (i, [vp, ctypes.c_longlong, vp]),
        "islbm_cnn_tanh_back": (i, [vp, vp, ctypes.c_longlong, vp]),
        "islbm_cnn_to_bf16": (i, [vp, vp, ctypes.c_longlong, vp]),
        "islbm_cnn_colsum": (i, [vp, vp, i, i, i, vp]),
        "islbm_cnn_mse": (i, [vp, vp, vp, i, vp, vp, i, ctypes.c_longlong, vp]),
        "islbm_cnn_pack_fields": (i, [vp, vp, vp, ctypes.c_longlong, d, d, d, vp, vp]),
        "islbm_cnn_unpack_fields": (i, [vp, ctypes.c_longlong, d, d, d, vp, vp, vp, vp]),
        "islbm_cnn_adam": (i, [vp, vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_longlong, vp]),
        "islbm_run_to_steady": (i, [h, d, ctypes.c_longlong, ctypes.c_longlong,
                                    P(ctypes.c_longlong), dp, dp]),
        "islbm_set_allocator": (i, [ALLOC_FN, FREE_FN, vp]),
        "islbm_set_row_range": (i, [h, i, i]),
        "islbm_get_rows": (i, [h, i, i, vp]),
        "islbm_set_rows": (i, [h, i, i, vp]),
        "islbm_reduce_sums": (i, [h, dp]),
        "islbm_finish_sums": (i, [h, dp, P(Reductions)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    # the library's device memory comes from torch's caching allocator when
    # torch has CUDA (else cudaMallocAsync on the owner's stream);
    # ISLBM_TORCH_ALLOCATOR=0 keeps the library's own default
    try:
        import torch
        if torch.cuda.is_available() and os.environ.get("ISLBM_TORCH_ALLOCATOR", "1") != "0":
            islbm_set_allocator(*torch_allocator())
    except ImportError:
        pass
    return lib


def _check(st: int, handle=None):
    if st != 0:
        msg = load_library().islbm_last_error(handle)
        raise IslbmError(st, msg.decode() if msg else "")


def _dptr(a):
    """Host double pointer of a C-contiguous float64 array (or None)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host(a, n):
    if a is None:
        return None
    arr = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr


def _check_tensor(t, n=None, name="tensor"):
    """Type, dtype, size (at least n values) and contiguity of a float64 tensor
    argument; None and plain ints (raw device addresses) pass unchecked."""
    if t is None or isinstance(t, int):
        return
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor or a device address, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: expected float64, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name}: needs at least {n} values, has {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")


def _devptr(t, n=None, name="tensor"):
    """Device address of a float64 CUDA tensor on the current device holding at
    least n values (checked here: the C side trusts its sizes).  A plain int is
    taken as a raw device address, unchecked."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    _check_tensor(t, n, name)
    if not t.is_cuda:
        raise ValueError(f"{name}: must live in CUDA device memory")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, but the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    return t.data_ptr()


def _handle_nodes(h) -> int:
    o = islbm_info(h)
    return int(o.n[0]) * int(o.n[1]) * (int(o.n[2]) if o.dim == 3 else 1)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# functions named as the C entry points
# ---------------------------------------------------------------------------

def islbm_mesh_uniform(n: int) -> np.ndarray:
    xi = np.empty(n + 2)
    _check(load_library().islbm_mesh_uniform(n, _dptr(xi)))
    return xi


def islbm_mesh_erf(n: int, a: float = 1.5) -> np.ndarray:
    xi = np.empty(n + 2)
    _check(load_library().islbm_mesh_erf(n, a, _dptr(xi)))
    return xi


def islbm_mesh_tanh(n: int, a: float = 1.5) -> np.ndarray:
    xi = np.empty(n + 2)
    _check(load_library().islbm_mesh_tanh(n, a, _dptr(xi)))
    return xi


def islbm_default_params() -> Params:
    p = Params()
    load_library().islbm_default_params(ctypes.byref(p))
    return p


def islbm_create(xi_x, xi_y, xi_z=None, Ra=1e6, Pr=0.71, lattice=None, precision="fp32",
                 params: Params | None = None, stream=None):
    lib = load_library()
    if lattice is None:
        lattice = "d2q9_d2q5" if xi_z is None else "d3q19_d3q7"
    xs = [np.ascontiguousarray(x, dtype=np.float64) if x is not None else None
          for x in (xi_x, xi_y, xi_z)]
    ns = [len(x) - 2 if x is not None else 0 for x in xs]
    h = ctypes.c_void_p()
    if stream is None:
        stream = _current_stream()
    st = lib.islbm_create(_dptr(xs[0]), ns[0], _dptr(xs[1]), ns[1], _dptr(xs[2]), ns[2],
                          float(Ra), float(Pr), LATTICES[lattice], PRECISIONS[precision],
                          ctypes.byref(params) if params is not None else None,
                          stream, ctypes.byref(h))
    _check(st)
    return h


def islbm_destroy(h):
    load_library().islbm_destroy(h)


def islbm_info(h) -> Info:
    o = Info()
    _check(load_library().islbm_info(h, ctypes.byref(o)), h)
    return o


def islbm_set_fields(h, T, u=None, v=None, w=None, rho=None, nodes=None):
    n = nodes if nodes is not None else int(np.asarray(T).size)
    arrs = [_host(a, n) for a in (rho, T, u, v, w)]
    _check(load_library().islbm_set_fields(h, *[_dptr(a) for a in arrs]), h)


def islbm_set_fields_device(h, T, u=None, v=None, w=None, rho=None):
    n = _handle_nodes(h)
    ptrs = [_devptr(a, n, k) for a, k in ((rho, "rho"), (T, "T"), (u, "u"), (v, "v"), (w, "w"))]
    _check(load_library().islbm_set_fields_device(h, *ptrs), h)


def islbm_set_populations(h, f, g):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    _check(load_library().islbm_set_populations(h, _dptr(f), _dptr(g)), h)


def islbm_step(h, n: int = 1):
    _check(load_library().islbm_step(h, int(n)), h)


def islbm_get_fields(h, shape, with_w=False, out=None):
    """Fields into new arrays, or into `out` (a dict of caller-owned contiguous
    float64 host arrays with the keys rho, T, u, v[, w], e.g. pinned memory)."""
    nodes = int(np.prod(shape))
    keys = ("rho", "T", "u", "v") + (("w",) if with_w else ())
    if out is None:
        out = {k: np.empty(nodes) for k in keys}
    flat = {}
    for k in keys:
        a = out[k]
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != nodes:
            raise ValueError(f"{k}: expected a contiguous float64 array of {nodes} values")
        flat[k] = a.reshape(-1)
    out = flat
    _check(load_library().islbm_get_fields(h, _dptr(out["rho"]), _dptr(out["T"]), _dptr(out["u"]),
                                           _dptr(out["v"]), _dptr(out.get("w"))), h)
    return {k: a.reshape(shape) for k, a in out.items()}


def islbm_get_fields_device(h, rho=None, T=None, u=None, v=None, w=None):
    n = _handle_nodes(h)
    ptrs = [_devptr(a, n, k) for a, k in ((rho, "rho"), (T, "T"), (u, "u"), (v, "v"), (w, "w"))]
    _check(load_library().islbm_get_fields_device(h, *ptrs), h)


def islbm_get_populations(h, q_flow, q_temp, shape):
    nodes = int(np.prod(shape))
    f = np.empty((q_flow, nodes))
    g = np.empty((q_temp, nodes))
    _check(load_library().islbm_get_populations(h, _dptr(f), _dptr(g)), h)
    return f.reshape((q_flow,) + tuple(shape)), g.reshape((q_temp,) + tuple(shape))


def islbm_reduce(h, check: bool = True) -> dict:
    r = Reductions()
    st = load_library().islbm_reduce(h, ctypes.byref(r))
    if check:
        _check(st, h)
    out = {k: getattr(r, k) for k, _ in Reductions._fields_}
    out["status"] = st
    return out


def islbm_set_row_range(h, row_begin: int, row_end: int):
    _check(load_library().islbm_set_row_range(h, int(row_begin), int(row_end)), h)


def _rows_buffer(buf, nbytes, name):
    """Address of a caller buffer of at least nbytes: a contiguous torch tensor
    (host or CUDA device) or numpy array."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            if not buf.is_contiguous():
                raise ValueError(f"{name}: must be contiguous")
            if buf.numel() * buf.element_size() < nbytes:
                raise ValueError(f"{name}: needs {nbytes} bytes, has "
                                 f"{buf.numel() * buf.element_size()}")
            if buf.is_cuda and buf.device.index != torch.cuda.current_device():
                raise ValueError(f"{name}: not on the current device")
            return buf.data_ptr()
    except ImportError:
        pass
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError(f"{name}: must be C-contiguous")
        if buf.nbytes < nbytes:
            raise ValueError(f"{name}: needs {nbytes} bytes, has {buf.nbytes}")
        return buf.ctypes.data
    raise TypeError(f"{name}: expected a torch tensor or a numpy array")


def rows_bytes(h, nrows: int) -> int:
    """Bytes of islbm_get_rows / islbm_set_rows for nrows rows of handle h."""
    o = islbm_info(h)
    elem = int(round(o.bytes_per_update / (2 * (o.q_flow + o.q_temp))))
    pitch = (int(o.n[0]) + 31) // 32 * 32
    return (o.q_flow + o.q_temp) * int(nrows) * pitch * elem


def islbm_get_rows(h, row0: int, nrows: int, dst):
    ptr = _rows_buffer(dst, rows_bytes(h, nrows), "dst")
    _check(load_library().islbm_get_rows(h, int(row0), int(nrows), ptr), h)


def islbm_set_rows(h, row0: int, nrows: int, src):
    ptr = _rows_buffer(src, rows_bytes(h, nrows), "src")
    _check(load_library().islbm_set_rows(h, int(row0), int(nrows), ptr), h)


def islbm_reduce_sums(h) -> np.ndarray:
    sums = np.zeros(REDUCTION_SUMS)
    _check(load_library().islbm_reduce_sums(h, _dptr(sums)), h)
    return sums


def islbm_finish_sums(h, sums, check: bool = True) -> dict:
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    if sums.size != REDUCTION_SUMS:
        raise ValueError(f"expected {REDUCTION_SUMS} sums, got {sums.size}")
    r = Reductions()
    st = load_library().islbm_finish_sums(h, _dptr(sums), ctypes.byref(r))
    if check:
        _check(st, h)
    out = {k: getattr(r, k) for k, _ in Reductions._fields_}
    out["status"] = st
    return out


def islbm_nusselt(h) -> dict:
    o = NuOut()
    _check(load_library().islbm_nusselt(h, ctypes.byref(o)), h)
    return {"vol": o.vol, "hot": o.hot, "cold": o.cold, "middle": o.middle}


def islbm_reynolds(h) -> float:
    x = ctypes.c_double()
    _check(load_library().islbm_reynolds(h, ctypes.byref(x)), h)
    return x.value


def islbm_mass(h) -> float:
    x = ctypes.c_double()
    _check(load_library().islbm_mass(h, ctypes.byref(x)), h)
    return x.value


def islbm_steady_change(h):
    du, dT = ctypes.c_double(), ctypes.c_double()
    _check(load_library().islbm_steady_change(h, ctypes.byref(du), ctypes.byref(dT)), h)
    return du.value, dT.value


def islbm_run_to_steady(h, tol=1e-9, interval=2000, max_steps=10_000_000, check=True):
    steps, du, dT = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    st = load_library().islbm_run_to_steady(h, float(tol), int(interval), int(max_steps),
                                             ctypes.byref(steps), ctypes.byref(du),
                                             ctypes.byref(dT))
    if check:
        _check(st, h)
    return {"steps": steps.value, "du": du.value, "dT": dT.value, "status": st}


def islbm_average_reset(h):
    _check(load_library().islbm_average_reset(h), h)


def islbm_average_add(h):
    _check(load_library().islbm_average_add(h), h)


def islbm_average_get(h, shape, with_w=False):
    """Time-averaged T, u, v (, w) and the number of states averaged."""
    nodes = int(np.prod(shape))
    out = {k: np.empty(nodes) for k in ("T", "u", "v")}
    if with_w:
        out["w"] = np.empty(nodes)
    count = ctypes.c_longlong()
    _check(load_library().islbm_average_get(h, _dptr(out["T"]), _dptr(out["u"]), _dptr(out["v"]),
                                            _dptr(out.get("w")), ctypes.byref(count)), h)
    return {k: a.reshape(shape) for k, a in out.items()}, count.value


def islbm_debug_bounds(reset=False) -> bool:
    """True if a bounds-checked build saw a staged index outside its window."""
    flagged = ctypes.c_int()
    _check(load_library().islbm_debug_bounds(1 if reset else 0, ctypes.byref(flagged)))
    return bool(flagged.value)


def islbm_selftest_wait_timeout(stream=None) -> int:
    """Status of the bounded-wait self-test (ISLBM_ERR_TIMEOUT = 6 is the expected outcome)."""
    if stream is None:
        stream = _current_stream()
    return load_library().islbm_selftest_wait_timeout(stream)


def islbm_selftest_wait_abort(stream=None):
    """(status, failed waits, ms) of the abort-flag self-test: ISLBM_ERR_TIMEOUT = 6,
    3 failed waits and about 1000 ms are the expected outcome."""
    if stream is None:
        stream = _current_stream()
    failed, ms = ctypes.c_int(), ctypes.c_int()
    st = load_library().islbm_selftest_wait_abort(stream, ctypes.byref(failed), ctypes.byref(ms))
    return st, failed.value, ms.value


def islbm_synchronize(h):
    _check(load_library().islbm_synchronize(h), h)


def islbm_save(h, path: str):
    _check(load_library().islbm_save(h, path.encode()), h)


def islbm_load(h, path: str):
    _check(load_library().islbm_load(h, path.encode()), h)


def islbm_reduce_noalloc(f, g, nx, ny, xi_x, xi_y, Ra, Pr=0.71, params: Params | None = None,
                         stream=None) -> dict:
    """Reductions of a 2-D state held in caller-owned device memory (torch CUDA
    float64 tensors or raw addresses); the library allocates nothing."""
    nx, ny = int(nx), int(ny)
    if nx < 1 or ny < 1:
        raise ValueError(f"nx, ny must be positive, got {nx}, {ny}")
    # the C side cannot see buffer sizes: check them (all four, then their
    # device) before anything is launched
    args = ((f, 9 * nx * ny, "f"), (g, 5 * nx * ny, "g"), (xi_x, nx + 2, "xi_x"),
            (xi_y, ny + 2, "xi_y"))
    for a in args:
        _check_tensor(*a)
    ptrs = tuple(_devptr(*a) for a in args)
    r = Reductions()
    if stream is None:
        stream = _current_stream()
    _check(load_library().islbm_reduce_noalloc(
        ptrs[0], ptrs[1], nx, ny, ptrs[2], ptrs[3], float(Ra),
        float(Pr), ctypes.byref(params) if params is not None else None, stream,
        ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in Reductions._fields_}


def islbm_autotune(n, mesh="tanh", a=1.5, precision="fp32", stream=None):
    """Fastest step-kernel variant of a square mesh and the per-variant step times (us)."""
    best = ctypes.c_int()
    us = (ctypes.c_double * KERNEL_VARIANTS)()
    if stream is None:
        stream = _current_stream()
    _check(load_library().islbm_autotune(int(n), MESH_KINDS[mesh], float(a), PRECISIONS[precision],
                                         stream, ctypes.byref(best), us))
    return best.value, list(us)


class _Member(object):
    """A batch member: the single-cavity calls on a handle owned by the batch."""


class Batch:
    """Many cavities advanced together (islbm_batch_*)."""

    def __init__(self, cavities, precision="fp32", autotune=False, params: Params | None = None,
                 stream=None):
        arr = (Cavity * len(cavities))()
        for k, c in enumerate(cavities):
            arr[k] = Cavity(int(c["n"]), MESH_KINDS[c.get("mesh", "tanh")], float(c.get("a", 1.5)),
                            float(c["Ra"]), float(c.get("Pr", 0.71)))
        h = ctypes.c_void_p()
        if stream is None:
            stream = _current_stream()
        _check(load_library().islbm_batch_create(len(cavities), arr, PRECISIONS[precision],
                                                 ctypes.byref(params) if params is not None else None,
                                                 1 if autotune else 0, stream, ctypes.byref(h)))
        self.h = h
        self.count = len(cavities)
        self.members = []
        for k in range(self.count):
            m = ctypes.c_void_p()
            _check(load_library().islbm_batch_member(self.h, k, ctypes.byref(m)))
            s = Solver.__new__(Solver)
            s.h = m
            s.owned = False
            s.info = islbm_info(m)
            s.dim = 2
            s.shape = (s.info.n[1], s.info.n[0])
            self.members.append(s)

    def tile_rows(self, k):
        return load_library().islbm_batch_tile_rows(self.h, k)

    def step(self, n=1):
        _check(load_library().islbm_batch_step(self.h, int(n)))

    def synchronize(self):
        _check(load_library().islbm_batch_synchronize(self.h))

    def run_to_steady(self, tol=1e-9, interval=2000, max_steps=10_000_000, check=True):
        steps = (ctypes.c_longlong * self.count)()
        st = load_library().islbm_batch_run_to_steady(self.h, float(tol), int(interval),
                                                      int(max_steps), steps)
        if check:
            _check(st)
        return list(steps), st

    def run_to_steady_nu(self, tol=1e-3, sample=1000, window=100, max_steps=10_000_000,
                         check=True):
        """islbm_batch_run_to_steady_nu: (steps, nu_mean, re_mean, status)."""
        steps = (ctypes.c_longlong * self.count)()
        nu = (ctypes.c_double * self.count)()
        re = (ctypes.c_double * self.count)()
        st = load_library().islbm_batch_run_to_steady_nu(self.h, float(tol), int(sample),
                                                         int(window), int(max_steps), steps, nu,
                                                         re)
        if check:
            _check(st)
        return list(steps), list(nu), list(re), st

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            load_library().islbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Solver:
    """One cavity solver handle; methods map one-to-one onto the C entry points."""

    def __init__(self, xi_x, xi_y, xi_z=None, Ra=1e6, Pr=0.71, precision="fp32",
                 params: Params | None = None, stream=None, **overrides):
        if overrides:
            params = params if params is not None else islbm_default_params()
            for k, v in overrides.items():
                if isinstance(v, str):
                    v = {"stencil": STENCILS, "kernel": KERNELS, "reference": REFERENCES}[k][v]
                setattr(params, k, v)
        self.h = islbm_create(xi_x, xi_y, xi_z, Ra, Pr, None, precision, params, stream)
        self.info = islbm_info(self.h)
        self.dim = self.info.dim
        n = list(self.info.n)
        self.shape = (n[1], n[0]) if self.dim == 2 else (n[2], n[1], n[0])

    def close(self):
        if getattr(self, "h", None) and getattr(self, "owned", True):
            islbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def time(self) -> int:
        return islbm_info(self.h).time

    def set_fields(self, T, u=None, v=None, w=None, rho=None):
        islbm_set_fields(self.h, T, u, v, w, rho, nodes=int(np.prod(self.shape)))

    def set_fields_device(self, T, u=None, v=None, w=None, rho=None):
        islbm_set_fields_device(self.h, T, u, v, w, rho)

    def set_populations(self, f, g):
        islbm_set_populations(self.h, f, g)

    def step(self, n: int = 1):
        islbm_step(self.h, n)

    def fields(self, out=None) -> dict:
        return islbm_get_fields(self.h, self.shape, with_w=self.dim == 3, out=out)

    def fields_device(self, rho=None, T=None, u=None, v=None, w=None):
        islbm_get_fields_device(self.h, rho, T, u, v, w)

    def average_reset(self):
        islbm_average_reset(self.h)

    def average_add(self):
        islbm_average_add(self.h)

    def average(self):
        return islbm_average_get(self.h, self.shape, with_w=self.dim == 3)

    def populations(self):
        return islbm_get_populations(self.h, self.info.q_flow, self.info.q_temp, self.shape)

    def reduce(self, check: bool = True) -> dict:
        return islbm_reduce(self.h, check)

    def synchronize(self):
        islbm_synchronize(self.h)

    def steady_change(self):
        return islbm_steady_change(self.h)

    def run_to_steady(self, tol=1e-9, interval=2000, max_steps=10_000_000, check=True):
        return islbm_run_to_steady(self.h, tol, interval, max_steps, check)

    def save(self, path):
        islbm_save(self.h, path)

    # ---- slab of a 2-D domain decomposition (paper_2509_01099_gb300.decomp) ----
    def set_row_range(self, row_begin: int, row_end: int):
        islbm_set_row_range(self.h, row_begin, row_end)

    def rows_bytes(self, nrows: int) -> int:
        return rows_bytes(self.h, nrows)

    def get_rows(self, row0: int, nrows: int, dst):
        islbm_get_rows(self.h, row0, nrows, dst)

    def set_rows(self, row0: int, nrows: int, src):
        islbm_set_rows(self.h, row0, nrows, src)

    def reduce_sums(self) -> np.ndarray:
        return islbm_reduce_sums(self.h)

    def finish_sums(self, sums, check: bool = True) -> dict:
        return islbm_finish_sums(self.h, sums, check)

    def load(self, path):
        islbm_load(self.h, path)

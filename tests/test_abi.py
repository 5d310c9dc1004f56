"""The C-ABI library: it builds, loads, exports every declared entry point, and its
host-side set-up agrees with the oracle.  No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2509_01099_gb300 as pkg
from paper_2509_01099_gb300 import build as B
from oracle import islbm_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pkg.load_library()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "islbm.h")).read()
    return sorted(set(re.findall(r"ISLBM_API\s+[\w\s\*]*?\b(islbm_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.EXPORTS)


@pytest.mark.parametrize("n", [4, 5, 64, 257, 1024])
def test_mesh_helpers_match_the_oracle(lib, n):
    np.testing.assert_allclose(pkg.islbm_mesh_erf(n, 1.5), O.mesh_erf(n, 1.5), rtol=0, atol=2e-16)
    np.testing.assert_allclose(pkg.islbm_mesh_tanh(n, 1.5), O.mesh_tanh(n, 1.5), rtol=0, atol=2e-16)
    np.testing.assert_allclose(pkg.islbm_mesh_uniform(n), O.mesh_uniform(n), rtol=0, atol=2e-16)
    xi = pkg.islbm_mesh_erf(n, 2.1)
    np.testing.assert_array_equal(xi + xi[::-1], np.ones_like(xi))


def test_mesh_helpers_reject_bad_arguments(lib):
    with pytest.raises(pkg.IslbmError):
        pkg.islbm_mesh_erf(3, 1.5)
    with pytest.raises(pkg.IslbmError):
        pkg.islbm_mesh_tanh(16, -1.0)


def test_default_params(lib):
    p = pkg.islbm_default_params()
    assert p.Ma == 0.1 and p.T_hot == 0.5 and p.T_cold == -0.5 and p.stencil == 0


def _create(xi_x, xi_y, **kw):
    return pkg.islbm_create(xi_x, xi_y, None, kw.pop("Ra", 1e6), 0.71, None, "fp32", None, None)


def test_create_validates_meshes_before_touching_a_device(lib):
    good = O.mesh_erf(16, 1.5)
    bad = good.copy()
    bad[5], bad[6] = bad[6], bad[5]                      # not increasing
    with pytest.raises(pkg.IslbmError) as e:
        _create(bad, good)
    assert e.value.status == 1
    with pytest.raises(pkg.IslbmError) as e:
        _create(O.mesh_erf(16, 1.5), O.mesh_erf(24, 1.5))  # different lattice units
    assert e.value.status == 1
    lopsided = good.copy()
    lopsided[-1] += 0.01                                  # ghost spacing differs at the ends
    with pytest.raises(pkg.IslbmError) as e:
        _create(lopsided, good)
    assert e.value.status == 1


def test_no_cpu_fallback_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    xi = O.mesh_erf(16, 1.5)
    with pytest.raises(pkg.IslbmError) as e:
        _create(xi, xi)
    assert e.value.status == 2                            # ISLBM_ERR_CUDA, loudly


def test_diffusivity_range_is_checked(lib):
    # tiny Ra on a coarse mesh gives alpha beyond the D2Q5 range (a_T > 1)
    xi = O.mesh_uniform(8)
    with pytest.raises(pkg.IslbmError) as e:
        _create(xi, xi, Ra=1e-4)
    assert e.value.status == 1


def test_kernel_variant_count_matches_header():
    import re
    from pathlib import Path
    from paper_2509_01099_gb300 import islbm as B
    text = (Path(__file__).resolve().parents[1] / "include" / "islbm.h").read_text()
    n = int(re.search(r"#define ISLBM_KERNEL_VARIANTS (\d+)", text).group(1))
    assert B.KERNEL_VARIANTS == n
    assert sorted(B.KERNELS.values()) == list(range(n))


def test_noalloc_binding_rejects_bad_tensors_before_any_launch():
    """The C side of islbm_reduce_noalloc cannot see buffer sizes: the binding
    checks dtype, size, contiguity and device first and raises (no assert, so
    `python -O` keeps the checks).  CPU tensors never reach the library."""
    import torch
    import paper_2509_01099_gb300 as pkg
    nx = ny = 8
    ok_f = torch.zeros(9 * nx * ny, dtype=torch.float64)
    ok_g = torch.zeros(5 * nx * ny, dtype=torch.float64)
    xi = torch.zeros(nx + 2, dtype=torch.float64)
    cases = [
        ((torch.zeros(9 * nx * ny - 1, dtype=torch.float64), ok_g, xi, xi), "f: needs at least"),
        ((ok_f, torch.zeros(5 * nx * ny - 1, dtype=torch.float64), xi, xi), "g: needs at least"),
        ((ok_f, ok_g, torch.zeros(nx + 1, dtype=torch.float64), xi), "xi_x: needs at least"),
        ((ok_f, ok_g, xi, torch.zeros(ny + 1, dtype=torch.float64)), "xi_y: needs at least"),
        ((ok_f.float(), ok_g, xi, xi), "f: expected float64"),
        ((ok_f, ok_g, xi, xi), "must live in CUDA device memory"),
    ]
    for args, msg in cases:
        with pytest.raises(ValueError, match=msg):
            pkg.islbm_reduce_noalloc(args[0], args[1], nx, ny, args[2], args[3], 1e6, 0.71)
    with pytest.raises(TypeError):
        pkg.islbm_reduce_noalloc([0.0], ok_g, nx, ny, xi, xi, 1e6, 0.71)


def test_allocator_registration_without_a_gpu():
    """islbm_set_allocator takes both callbacks or neither; registering does
    not touch the device."""
    import paper_2509_01099_gb300 as pkg
    from paper_2509_01099_gb300 import islbm as I
    lib = pkg.load_library()
    calls = []
    pkg.islbm_set_allocator(lambda n, d, s: calls.append(n) or 0, lambda p, d, s: None)
    assert calls == []
    # one function alone is an argument error
    assert lib.islbm_set_allocator(I.ALLOC_FN(lambda *a: None), I.FREE_FN(), None) != 0
    pkg.islbm_set_allocator(None, None)
    # every callback ever registered stays referenced (handles keep theirs)
    assert len(I._allocator_refs) >= 2


def test_fp16neq_needs_the_2d_pipelined_kernels(lib):
    """The non-equilibrium storage is decoded per staged tile: only the 2-D
    pipelined kernels with 8-row tiles run it.  Every other choice is refused
    before a device is touched."""
    xi = O.mesh_tanh(16, 1.5)
    cases = [dict(xi_z=xi), dict(kernel=1), dict(kernel=2), dict(kernel=3), dict(kernel=6),
             dict(stencil=1)]
    for kw in cases:
        p = pkg.islbm_default_params()
        p.kernel = kw.get("kernel", 0)
        p.stencil = kw.get("stencil", 0)
        with pytest.raises(pkg.IslbmError) as e:
            pkg.islbm_create(xi, xi, kw.get("xi_z"), 1e6, 0.71, None, "fp16neq", p, None)
        assert e.value.status == 1, kw

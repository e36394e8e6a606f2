"""The C ABI library builds, loads and exports every symbol the header declares.
CPU only: no call here touches a GPU (only argument checks that fail before
any CUDA call)."""

import ctypes
import os

import pytest

import paper_2501_14911_gb300 as bti

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(bti.lib_path()):
        from paper_2501_14911_gb300 import build

        build.build()
    return bti.lib()


def test_header_declares_the_hot_path_calls():
    names = bti.header_symbols()
    for n in ("bti_create", "bti_destroy", "bti_set_blocks", "bti_set_prior_se_grid", "bti_set_noise",
              "bti_apply_F", "bti_apply_FT", "bti_apply_Fq", "bti_apply_Gstar", "bti_build_K",
              "bti_factor_K", "bti_infer_map", "bti_predict_qoi", "bti_sync", "bti_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(L):
    for name in bti.header_symbols():
        assert hasattr(L, name), f"{name} declared in include/bti.h but not exported"


def test_version_string(L):
    assert L.bti_version().decode().startswith("libbti")


def test_host_side_argument_errors_need_no_gpu(L):
    h = ctypes.c_void_p()
    # sizes are validated before any CUDA call
    assert L.bti_create(0, 4, 0, 8, 0, None, ctypes.byref(h)) == 1
    assert L.bti_create(16, -1, 0, 8, 0, None, ctypes.byref(h)) == 1
    assert L.bti_create(16, 4, 0, 0, 0, None, ctypes.byref(h)) == 1
    assert L.bti_create(16, 4, 0, 4096, 0, None, ctypes.byref(h)) == 1  # L = 8192 > 4096
    assert L.bti_create(16, 4, 0, 8, 0, None, None) == 1
    assert not h.value
    assert L.bti_destroy(None) == 1
    assert L.bti_sync(None) == 1
    assert L.bti_apply_F(None, None, None, 1, 0) == 1
    assert L.bti_last_error(None).decode() == "null handle"


def test_no_cpu_fallback_in_binding():
    """The binding module contains no numeric fallback: every Handle method calls the library."""
    src = open(os.path.join(ROOT, "paper_2501_14911_gb300", "_binding.py")).read()
    for forbidden in ("numpy", "torch.fft", "oracle", "@ ", "matmul", "einsum"):
        assert forbidden not in src, forbidden

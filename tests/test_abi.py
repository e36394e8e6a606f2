"""The C ABI library builds, loads and exports every symbol the header declares, and the
binding's ctypes signatures match the header's prototypes.
CPU only: no call here touches a GPU (only argument checks that fail before
any CUDA call)."""

import ctypes
import os
import re

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


def _c_kind(param):
    """Argument class of one C parameter: pointer, 64- or 32-bit integer, or double."""
    p = " ".join(param.split())
    if "*" in p or p.startswith("bti_handle"):
        return "ptr"
    return {"int64_t": "i64", "int": "i32", "double": "f64", "bti_op": "i32", "bti_prec": "i32"}[p.rsplit(" ", 1)[0]]


def _py_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    if t is ctypes.c_double:
        return "f64"
    return {8: "i64", 4: "i32"}[ctypes.sizeof(t)]


def test_binding_argtypes_match_the_header_prototypes(L):
    """A ctypes signature that disagrees with the C prototype (an int where the C side takes
    int64_t, a scalar where it takes a pointer) would corrupt arguments without an error."""
    with open(os.path.join(ROOT, "include", "bti.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    protos = re.findall(r"^\s*(bti_status|const char\s*\*)\s+(bti_\w+)\s*\(([^)]*)\)\s*;", text, re.M)
    assert {name for _, name, _ in protos} == set(bti.header_symbols())
    for ret, name, params in protos:
        params = [q for q in (x.strip() for x in params.split(",")) if q and q != "void"]
        fn = getattr(L, name)
        assert fn.argtypes is not None, f"{name}: the binding sets no argtypes"
        assert [_c_kind(q) for q in params] == [_py_kind(t) for t in fn.argtypes], name
        assert fn.restype is (ctypes.c_int if ret == "bti_status" else ctypes.c_char_p), name


def test_binding_constants_and_struct_match_the_header():
    """The enum values, the kernel classes of the profile hook and bti_solve_info's layout as
    the binding mirrors them."""
    from paper_2501_14911_gb300 import _binding as b

    with open(os.path.join(ROOT, "include", "bti.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(BTI_\w+)\s*=\s*(\d+)", text)}
    assert (b.OP_F, b.OP_G, b.OP_FQ) == (enum["BTI_OP_F"], enum["BTI_OP_G"], enum["BTI_OP_FQ"])
    assert (b.F64, b.F32, b.DF64, b.F16) == tuple(enum["BTI_P_" + t] for t in ("F64", "F32", "DF64", "F16"))
    assert b.STATUS == {v: k for k, v in enum.items() if k == "BTI_OK" or k.startswith("BTI_ERR_")}
    kcls = ["RFFT", "PROD_FWD", "REDUCE", "IRFFT", "PROD_ADJ", "DENSE"]
    assert len(b.KCLASSES) == enum["BTI_K_NCLASS"]
    assert [enum["BTI_K_" + k] for k in kcls] == list(range(len(kcls)))
    assert list(b.KCLASSES) == [k.lower() for k in kcls]
    body = re.search(r"typedef struct \{([^}]*)\} bti_solve_info;", text).group(1)
    fields = [tuple(x.split()) for x in body.replace("\n", " ").split(";") if x.strip()]
    ct = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [(n, ct[t]) for t, n in fields] == list(b.SolveInfo._fields_)

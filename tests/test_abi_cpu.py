"""CPU-only checks of the C-ABI library: it loads, it exports every function include/*.h declares,
and argument validation that happens before any CUDA call reports the documented status."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2602_12011_gb300 import _lib as L
from paper_2602_12011_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions(header_glob="pespace_gb300.h"):
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", header_glob)):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?(pe_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pe_create_detector", "pe_destroy_detector", "pe_set_data_psd", "pe_loglike_batch",
              "pe_loglike_grad_batch", "pe_fisher", "pe_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_test_build_exports_its_header_and_the_product_does_not(lib):
    """include/pespace_gb300_test.h is exported by the test build (fault injection, index checks)
    alongside the whole product boundary, and by nothing the product library loads."""
    test_names = declared_functions("pespace_gb300_test.h")
    assert test_names and all(n.startswith("pe_test_") for n in test_names)
    tlib = C.CDLL(B.build(variant="test"))
    assert not [n for n in test_names + declared_functions() if not hasattr(tlib, n)]
    assert not [n for n in test_names if hasattr(lib, n)]
    tlib.pe_test_fault_arm.argtypes = [C.c_int, C.c_long]
    tlib.pe_test_fault_count.argtypes = [C.c_int]
    tlib.pe_test_fault_count.restype = C.c_long
    assert tlib.pe_test_fault_arm(3, 1) == L.PE_EINVAL
    assert tlib.pe_test_fault_arm(0, -1) == L.PE_EINVAL
    assert tlib.pe_test_fault_arm(-1, 0) == L.PE_OK
    assert tlib.pe_test_fault_count(7) == -1


def test_abi_version(lib):
    assert L.pe_abi_version() == 1


def test_null_arguments_are_einval_without_cuda(lib):
    h = C.c_void_p()
    assert lib.pe_create_detector(None, 1.0, 1, 1, C.byref(h)) == L.PE_EINVAL
    assert b"NULL" in lib.pe_last_error()
    cfg = L.config_from_dict(dict(orbit=0, arm_m=2.5e9, oms_m_rtHz=1e-11, acc_ms2_rtHz=1e-15, tdi_gen=17))
    assert lib.pe_create_detector(C.byref(cfg), 1.0, 1, 1, C.byref(h)) == L.PE_EINVAL
    assert b"tdi_gen" in lib.pe_last_error()
    assert lib.pe_loglike_batch(None, 1, None, 1, 1, None, None, None, None) == L.PE_EINVAL
    assert lib.pe_destroy_detector(None) == L.PE_OK
    # tuning entry points: handle checks come before any device work
    assert lib.pe_tune_set(None, 1, 1, 0x1F, 0, 8, 1) == L.PE_EINVAL
    assert lib.pe_autotune(None, 1, None, 1, 0x1F, None, None, None, None) == L.PE_EINVAL


def test_product_binding_never_imports_the_oracle():
    """The product path (package sources) must not reach the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_12011_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(path).read()
            assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or path.endswith("workloads.py"), path


@pytest.mark.parametrize("T,mask,nbins", [(2.0 ** 17, 0x1F, 64), (2.0 ** 22, 0x1F, 256), (2.0 ** 20, 0x01, 128)])
def test_hetero_default_edges_match_the_oracle(lib, oracle_mod, T, mask, nbins):
    """pe_hetero_default_edges is host code (no GPU): the same edges as the oracle's construction."""
    import numpy as np
    from oracle import hetero as HT
    from paper_2602_12011_gb300 import workloads as W
    k0, nb = W.grid(T)
    th0 = W.theta_injection(T)
    mine = L.pe_hetero_default_edges(T, k0, nb, th0, mask, nbins)
    ref = HT.default_edges(T, k0, nb, th0, mask, nbins)
    assert np.array_equal(mine, ref)


def test_hetero_argument_errors_without_cuda(lib):
    import numpy as np
    th = np.array([1e6, 2, 0, 0, 1, 0, 0, 0, 0, 0, 0.0])
    with pytest.raises(L.PeError) as e:
        L.pe_hetero_default_edges(2.0 ** 16, 7, 3000, th, 0x40, 32)
    assert e.value.status == L.PE_EINVAL
    out = np.zeros(2, dtype=np.int64)
    n = C.c_int(2)
    assert lib.pe_hetero_default_edges(2.0 ** 16, 7, 3000, L._ptr(th), 0x1F, 32, L._ptr(out), C.byref(n)) == L.PE_EINVAL
    assert b"do not fit" in lib.pe_last_error()
    h = C.c_void_p()
    assert lib.pe_hetero_create(None, None, 0x1F, None, 0, C.byref(h)) == L.PE_EINVAL
    assert lib.pe_hetero_loglike_batch(None, 1, None, 1, None, None, None, None) == L.PE_EINVAL
    assert lib.pe_hetero_destroy(None) == L.PE_OK


def test_wait_limit_without_cuda(lib):
    """The bounded host wait's limit (PE_ETIMEOUT past it) is set and read without a GPU."""
    old = L.pe_get_wait_limit()
    assert old > 0
    try:
        L.pe_set_wait_limit(2.5)
        assert L.pe_get_wait_limit() == 2.5
        for bad in (0.0, -1.0, float("inf"), float("nan")):
            with pytest.raises(L.PeError) as e:
                L.pe_set_wait_limit(bad)
            assert e.value.status == L.PE_EINVAL
        assert L.pe_get_wait_limit() == 2.5
    finally:
        L.pe_set_wait_limit(old)

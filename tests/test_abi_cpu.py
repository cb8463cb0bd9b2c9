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


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
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


def test_product_binding_never_imports_the_oracle():
    """The product path (package sources) must not reach the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_12011_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(path).read()
            assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or path.endswith("workloads.py"), path

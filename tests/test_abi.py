"""The C-ABI library loads and exports every entry point that include/bqs.h declares.

No compute calls: these run without a GPU.  Argument checks that return before
any CUDA call are exercised too.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bqs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1604_06697_gb300 import _native, build
    build.build()
    return _native.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bqs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bqs_partition", "bqs_sort", "bqs_sort_segmented", "bqs_sort_pairs",
                     "bqs_set_option", "bqs_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1604_06697_gb300 import _native
    assert set(declared_functions()) == set(_native.SIGNATURES)


def test_argument_checks_without_gpu(lib):
    from paper_1604_06697_gb300 import _native
    assert lib.bqs_sort(None, 0, 0, None) == 0          # empty: no-op
    assert lib.bqs_sort(None, 1, 0, None) == 0          # one key: no-op
    assert lib.bqs_sort(None, -1, 0, None) == -1
    assert lib.bqs_sort(None, 10, 7, None) == -1        # bad dtype
    assert lib.bqs_sort(ctypes.c_void_p(8), 10, 0, None) == -1   # misaligned
    assert lib.bqs_sort(None, 1 << 33, 0, None) == -1   # beyond 32-bit counts
    assert lib.bqs_sort_segmented(None, None, 0, 0, None) == 0
    assert lib.bqs_sort_segmented(None, None, 3, 0, None) == -1
    pv = _native.Pivot()
    pv.dtype, pv.reserved = 0, 0
    split = ctypes.c_int64(5)
    assert lib.bqs_partition(None, 0, ctypes.byref(pv), None, ctypes.byref(split), None) == 0
    assert split.value == 0
    pv.reserved = 1
    assert lib.bqs_partition(None, 0, ctypes.byref(pv), None, ctypes.byref(split), None) == -1
    assert lib.bqs_status_string(-1) == b"invalid argument"


def test_options_round_trip(lib):
    import paper_1604_06697_gb300 as bqs
    old = bqs.get_option("small_cutoff")
    try:
        bqs.set_option("small_cutoff", 64)
        assert bqs.get_option("small_cutoff") == 64
        bqs.set_option("small_cutoff", 4096)       # key-only sorts; key-value clamp to 2048
        assert bqs.get_option("small_cutoff") == 4096
        with pytest.raises(bqs.BqsError):
            bqs.set_option("small_cutoff", 4097)
        with pytest.raises(bqs.BqsError):
            bqs.set_option("small_cutoff", 1)
        with pytest.raises(bqs.BqsError):
            bqs.set_option("pivot", 7)             # rules 0..6 (Sec. 4)
        old_pivot = bqs.get_option("pivot")
        for rule in range(7):
            bqs.set_option("pivot", rule)
            assert bqs.get_option("pivot") == rule
        bqs.set_option("pivot", old_pivot)
        old_ls = bqs.get_option("local_sort")
        assert old_ls == 0                          # default: leaves go to the network kernels
        for v in (0, 1, 128):
            bqs.set_option("local_sort", v)
            assert bqs.get_option("local_sort") == v
        with pytest.raises(bqs.BqsError):
            bqs.set_option("local_sort", 129)
        bqs.set_option("local_sort", old_ls)
    finally:
        bqs.set_option("small_cutoff", old)


def test_workspace_bytes_grows_with_n(lib):
    import paper_1604_06697_gb300 as bqs
    a = bqs.workspace_bytes(1 << 20, "int32")
    b = bqs.workspace_bytes(1 << 22, "int32")
    assert b > a >= 4 * (1 << 20)
    assert bqs.workspace_bytes(1 << 20, "int64", with_payload=True) >= 12 * (1 << 20)


def test_oracle_and_product_share_no_code():
    prod = os.path.join(ROOT, "paper_1604_06697_gb300")
    for dirpath, _, files in os.walk(prod):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "bqs_oracle" not in text, f
    text = open(os.path.join(ROOT, "oracle", "bqs_oracle.cpp")).read()
    assert "#include \"bqs" not in text and "bqs_common" not in text
    text = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert not re.search(r"^\s*(import|from)\s+(paper_1604_06697_gb300|\.)", text, re.M)

"""The C-ABI library loads and exports every function include/mm.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(mm_[a-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1306_6192_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mm_init", "mm_gemm", "mm_gemm_grouped", "mm_submit", "mm_poll",
                     "mm_shutdown", "mm_check", "mm_strerror"):
        assert required in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(built_lib, name):
    assert hasattr(built_lib, name), name


def test_binding_has_every_name():
    import paper_1306_6192_gb300 as mm
    for name in declared_functions():
        assert hasattr(mm, name), name


def test_strerror_without_gpu(built_lib):
    import paper_1306_6192_gb300 as mm
    assert mm.mm_strerror(mm.MM_OK) == "ok"
    assert "budget" in mm.mm_strerror(mm.MM_EBUDGET)


def test_calls_before_init_report_it(built_lib):
    """Entry points that need the device return MM_ENOTINIT before mm_init,
    without touching CUDA (no GPU here)."""
    import paper_1306_6192_gb300 as mm
    if mm.mm_sync(None) != mm.MM_ENOTINIT:
        pytest.skip("the library was initialised by an earlier test in this process")
    F32, SPLIT = mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3
    assert mm.mm_gemm(8, 8, 8, 1, 1, 1, F32, SPLIT) == mm.MM_ENOTINIT
    assert mm.mm_gemm_axpby(8, 8, 8, 1.0, 1, 1, -1.0, 1, 1, F32, SPLIT) == mm.MM_ENOTINIT
    assert mm.mm_gemm_axpby_async(8, 8, 8, 1.0, 1, 1, -1.0, 1, 1, F32, SPLIT) == mm.MM_ENOTINIT
    assert mm.mm_add(8, 8, 1.0, 1, 1.0, 1, 1, F32) == mm.MM_ENOTINIT

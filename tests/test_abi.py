"""The C ABI library builds, loads without a GPU, and exports every symbol that
include/geotrace.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gt_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2310_15183_gb300 import build, geotrace
    build.build()
    return geotrace.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2310_15183_gb300 import geotrace
    declared = _declared()
    assert "gt_trace" in declared and "gt_set_camera" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(geotrace.EXPORTS)


def test_strerror_is_total(lib):
    for code in range(-8, 2):
        assert isinstance(lib.gt_strerror(code), bytes)


def test_null_arguments_rejected_without_device(lib):
    """Argument checks that need no device answer GT_ERR_INVALID_ARG."""
    assert lib.gt_create(None, 0, None) == -1
    assert lib.gt_destroy(None) == -1
    assert lib.gt_set_spacetime(None, 0.5, 0.0, 0.0) == -1
    assert lib.gt_trace(None, 10, 1e-4, 0, None, None, None, None, None, None) == -1


def test_library_is_sm103a_only():
    """The build passes exactly one -gencode, for sm_103a."""
    from paper_2310_15183_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2310_15183_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "geodesic_oracle" not in src, fn

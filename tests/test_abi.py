"""CPU checks of the C ABI: the library builds, loads, exports every symbol
include/bhtree.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as bh
    return bh.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "bhtree.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    import paper_1112_4539_gb300 as bh
    names = _declared()
    assert len(names) >= 12, names
    for name in names:
        assert hasattr(L, name), name
    assert set(bh.SYMBOLS) <= set(names)


def test_version_and_strerror(L):
    assert L.bh_version() >= 10000
    for code in range(0, -9, -1):
        s = L.bh_strerror(code).decode()
        assert s and s != "unknown error"
    assert L.bh_strerror(-99).decode() == "unknown error"


def test_config_defaults(L):
    import paper_1112_4539_gb300 as bh
    c = bh.config()
    assert (c.leaf_size, c.group_size, c.order, c.fp64_node_threshold, c.block_threads) == (8, 64, 1, 4096, 128)


@pytest.mark.parametrize("field,value", [("leaf_size", 0), ("leaf_size", 65), ("group_size", 0),
                                         ("group_size", 257), ("order", 3), ("block_threads", 96),
                                         ("fp64_node_threshold", 0)])
def test_create_rejects_bad_config(L, field, value):
    import paper_1112_4539_gb300 as bh
    c = bh.config(**{field: value})
    h = ctypes.c_void_p()
    assert L.bh_create(ctypes.byref(h), ctypes.byref(c), 1000, 0) == bh.BH_ERR_INVALID
    assert not h.value


def test_create_rejects_bad_sizes(L):
    import paper_1112_4539_gb300 as bh
    h = ctypes.c_void_p()
    assert L.bh_create(ctypes.byref(h), None, 0, 0) == bh.BH_ERR_INVALID
    assert L.bh_create(ctypes.byref(h), None, 1 << 30, 0) == bh.BH_ERR_TOO_LARGE
    assert L.bh_create(None, None, 10, 0) == bh.BH_ERR_INVALID


def test_null_context_and_args(L):
    import paper_1112_4539_gb300 as bh
    assert L.tree_build(None, None, 10, None) == bh.BH_ERR_INVALID
    assert L.tree_moments(None, ctypes.c_float(0.5), None) == bh.BH_ERR_INVALID
    assert L.tree_force(None, ctypes.c_float(0.01), None, None) == bh.BH_ERR_INVALID
    assert L.bh_status(None, None) == bh.BH_ERR_INVALID
    assert L.bh_selftest_wait(None, bh.SELFTEST_TILE_RING, None) == bh.BH_ERR_INVALID
    # direct_force validates sizes, precision and eps before any CUDA call
    assert L.direct_force(None, -1, None, None, 1, 0.0, None, 32, None) == bh.BH_ERR_INVALID
    assert L.direct_force(None, 1, None, None, 1, 0.0, None, 16, None) == bh.BH_ERR_INVALID
    assert L.direct_force(None, 1, None, None, 1, -1.0, None, 32, None) == bh.BH_ERR_INVALID
    assert L.direct_force(None, 1 << 31, None, None, 1, 0.0, None, 32, None) == bh.BH_ERR_TOO_LARGE
    assert L.direct_force(None, 0, None, None, 0, 0.0, None, 32, None) == bh.BH_OK


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1112_4539_gb300 as bh
    monkeypatch.setattr(bh, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bh, "_lib", None)
    with pytest.raises(ImportError):
        bh.lib()


def test_product_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1112_4539_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt and "liboracle" not in txt, f

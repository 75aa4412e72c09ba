"""The C ABI on a machine without a GPU: the library loads, exports every declared symbol, and rejects invalid
forests on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_08063_gb300.build import build
    build()
    from paper_2403_08063_gb300 import _lib
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "octmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_2403_08063_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES)


def _create(lib, R, n, keys):
    from paper_2403_08063_gb300 import _lib
    arr = np.ascontiguousarray([(0, *k) for k in keys], dtype=np.int32)
    cfg = _lib.MGConfig()
    cfg.roots, cfg.n, cfg.n_leaves = R, n, len(keys)
    cfg.leaves = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cfg.coeff, cfg.interface_flux, cfg.precision, cfg.nu1, cfg.nu2, cfg.max_coarse = 0, 1, 0, 2, 2, 512
    cfg.inner_cycles = 1
    cfg.n_problems = 1
    h = ctypes.c_void_p()
    st = lib.mg_forest_create(ctypes.byref(cfg), ctypes.byref(h))
    return st, h, lib.mg_last_error().decode()


def test_rejects_bad_block_size(lib):
    st, h, msg = _create(lib, 2, 6, [(0, i, j, k) for k in range(2) for j in range(2) for i in range(2)])
    assert st == 3 and h.value is None and "power of two" in msg


def test_rejects_unbalanced_forest(lib):
    # root (0,0,0) refined three times next to its face x = 1/2: a level-3 block touches the level-0 root (1,0,0)
    import synthetic as syn
    keys = syn.refine_box(2, (0.45, 0.0, 0.0), (0.5, 0.05, 0.05), 3)
    st, h, msg = _create(lib, 2, 8, keys)
    assert st == 2 and "balanced" in msg


def test_rejects_holes_and_overlaps(lib):
    keys = [(0, i, j, k) for k in range(2) for j in range(2) for i in range(2)][:-1]
    st, _, msg = _create(lib, 2, 8, keys)
    assert st == 2 and "cover" in msg
    keys = [(0, i, j, k) for k in range(2) for j in range(2) for i in range(2)] + [(1, 0, 0, 0)]
    st, _, msg = _create(lib, 2, 8, keys)
    assert st == 2 and "overlap" in msg


def test_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.mg_forest_create(None, ctypes.byref(h)) == 1

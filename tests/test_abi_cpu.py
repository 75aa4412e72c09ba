"""The C ABI on a machine without a GPU: the library loads, exports every declared symbol, the ctypes binding
agrees with the header (argument kinds, the config struct's layout), and invalid forests are rejected on the host
before the device is touched."""
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


def _prototypes():
    text = open(os.path.join(ROOT, "include", "octmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\s*\b(mg_[a-z_]+)\s*\(([^)]*)\)\s*;", text):
        params = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        out[name] = (ret.split()[-1] if "*" not in ret else "*", params)
    return out


def _c_kind(decl):
    if "*" in decl:
        return "ptr"
    for word, kind in (("double", "f64"), ("int64_t", "i64"), ("int32_t", "i32"), ("mg_status", "i32")):
        if re.search(rf"\b{word}\b", decl):
            return kind
    raise AssertionError(f"unknown C type in {decl!r}")


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    return {ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_double: "f64"}[t]


def test_binding_signatures_match_the_header():
    """Every prototype in the header and its ctypes declaration agree in arity and in the kind of every argument
    and result (pointer, int32, int64, double), so no call marshals an argument into the wrong register."""
    from paper_2403_08063_gb300 import _lib
    protos = _prototypes()
    assert set(protos) == set(_lib.SIGNATURES)
    for name, (ret, params) in protos.items():
        res, args = _lib.SIGNATURES[name]
        want_ret = "void" if ret == "void" else ("ptr" if ret == "*" else _c_kind(ret))
        assert _ctypes_kind(res) == want_ret, name
        assert [_c_kind(p) for p in params] == [_ctypes_kind(a) for a in args], name


def test_config_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirror of mg_config has the C compiler's field offsets and size (a mismatch would let the library
    read the caller's fields at the wrong places)."""
    import shutil
    import subprocess
    from paper_2403_08063_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in _lib.MGConfig._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"octmg.h\"\nint main(void) {\n"
                   + "".join(f'    printf("%zu\\n", offsetof(mg_config, {f}));\n' for f in fields)
                   + '    printf("%zu\\n", sizeof(mg_config));\n    return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [getattr(_lib.MGConfig, f).offset for f in fields] + [ctypes.sizeof(_lib.MGConfig)]
    assert got == want, list(zip(fields + ["sizeof"], got, want))


def _create_rows(lib, rows, R=2, n=8, **fields):
    """mg_forest_create with leaf rows (problem, level, i, j, k) and config fields overridden."""
    from paper_2403_08063_gb300 import _lib
    arr = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 5)
    cfg = _lib.MGConfig()
    cfg.roots, cfg.n, cfg.n_leaves = R, n, len(arr)
    cfg.leaves = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cfg.coeff, cfg.interface_flux, cfg.precision, cfg.nu1, cfg.nu2, cfg.max_coarse = 0, 1, 0, 2, 2, 512
    cfg.inner_cycles, cfg.n_problems = 1, 1
    for name, value in fields.items():
        setattr(cfg, name, value)
    h = ctypes.c_void_p()
    st = lib.mg_forest_create(ctypes.byref(cfg), ctypes.byref(h))
    assert h.value is None
    return st, lib.mg_last_error().decode()


_ROOTS = [(0, 0, i, j, k) for k in range(2) for j in range(2) for i in range(2)]


@pytest.mark.parametrize("rows,fields,status,text", [
    (_ROOTS, {"n_leaves": 0}, 1, "null config"),
    (_ROOTS, {"coeff": 2}, 1, "bad coeff"),
    (_ROOTS, {"nu1": 0, "nu2": 0}, 1, "nu1"),
    (_ROOTS, {"interface_flux": -1}, 1, "interface_flux"),
    (_ROOTS, {"c2f_variant": 3}, 1, "c2f_variant"),
    (_ROOTS, {"omega": 2.5}, 1, "omega"),
    (_ROOTS, {"omega": float("nan")}, 1, "omega"),
    (_ROOTS, {"coarse_iters": -1}, 1, "coarse_iters"),
    (_ROOTS, {"coarse_coef": 2}, 1, "coarse_coef"),
    (_ROOTS, {"prolongation": 2}, 1, "prolongation"),
    (_ROOTS, {"smoother": 1, "precision": 1}, 1, "damped Jacobi"),
    (_ROOTS, {"roots": 0}, 1, "roots must be"),
    (_ROOTS, {"n": 2048}, 3, "4..1024"),
    (_ROOTS[:-1] + [(1, 0, 1, 1, 1)], {}, 1, "problem index"),
    (_ROOTS[:-1] + [(0, 0, 2, 1, 1)], {}, 2, "outside the domain"),
    (_ROOTS + [_ROOTS[3]], {}, 2, "duplicate"),
    (_ROOTS, {"n_problems": 2}, 2, "(problem 1)"),
    ([(0, 20, 0, 0, 0)], {}, 1, "too deep"),
])
def test_host_checks_reject_each_bad_config(lib, rows, fields, status, text):
    """Every config and leaf check runs on the host before any device call, with its own status and message."""
    st, msg = _create_rows(lib, rows, **fields)
    assert st == status and text in msg, (st, msg)


def test_batch_host_checks(lib):
    from paper_2403_08063_gb300 import _lib
    rows = np.ascontiguousarray([(p, 0, 0, 0, 0) for p in range(3)], dtype=np.int32)
    cfg = _lib.MGConfig()
    cfg.roots, cfg.n, cfg.n_leaves, cfg.n_problems = 1, 8, 3, 3
    cfg.coeff, cfg.interface_flux, cfg.precision, cfg.nu1, cfg.nu2 = 1, 1, 1, 2, 2
    h = ctypes.c_void_p()
    assert lib.mg_batch_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1  # no leaves
    cfg.leaves = rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    pn = np.ascontiguousarray([8, 6, 16], dtype=np.int32)
    st = lib.mg_batch_create(ctypes.byref(cfg), pn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(h))
    assert st == 3 and "problem 1" in lib.mg_last_error().decode() and h.value is None
    m = ctypes.c_int32()
    assert lib.mg_batch_set_tail_mode(None, 0) == 1 and lib.mg_batch_get_tail_mode(None, ctypes.byref(m)) == 1
    assert lib.mg_alu_peaks(None, None) == 1  # no output: refused before any CUDA call


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the binding raises instead of computing anything."""
    from paper_2403_08063_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "libocmg.so"))


def test_product_code_never_touches_the_oracle():
    """The package and the header name neither the oracle module nor its functions."""
    pkg = os.path.join(ROOT, "paper_2403_08063_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"\boracle\b|octree_mg|OracleMG", text), name

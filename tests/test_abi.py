"""Host-side checks of the C ABI: the library builds/loads and exports every
function declared in include/ssnal_en.h; the ctypes structs match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(ssnal_en_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_03970_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    import paper_2006_03970_gb300 as pkg
    for n in _declared():
        assert n in pkg.EXPORTS, n
        if n != "ssnal_en_status_string":
            assert hasattr(pkg, n), n


def test_struct_layouts(lib):
    import paper_2006_03970_gb300 as pkg
    # sizes implied by the header's field lists (LP64)
    assert ctypes.sizeof(pkg.Matrix) == 3 * 8 + 2 * 4 + 3 * 8
    assert ctypes.sizeof(pkg.Options) == 6 * 8 + 8 * 4 + 8 + 2 * 4 + 8 + 8
    assert ctypes.sizeof(pkg.Result) == 4 * 4 + 8 + 8 * 8 + 2 * 4
    assert ctypes.sizeof(pkg.Instance) == 6 * 8
    assert ctypes.sizeof(pkg.TunePoint) == 5 * 8
    assert ctypes.sizeof(pkg.BatchFit) == 8 * 8


def test_default_options_without_gpu(lib):
    import paper_2006_03970_gb300 as pkg
    o = pkg.ssnal_en_default_options()
    assert (o.sigma0, o.sigma_growth, o.mu, o.tol, o.max_ls, o.ls_fused) == (5e-3, 5.0, 0.2, 1e-6, 40, 16)
    lib.ssnal_en_status_string.restype = ctypes.c_char_p
    assert lib.ssnal_en_status_string(3) == b"iteration limit reached before the KKT tolerance"


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    import paper_2006_03970_gb300 as pkg
    L = pkg.load_library()
    ctx = ctypes.c_void_p()
    assert L.ssnal_en_create(ctypes.byref(ctx), None, None, None) == pkg.EINVAL
    bad = pkg.Matrix(m=10, n=5, lda=9, dtype=0, reserved=0, data=16, col_mean=None, col_scale=None)
    assert L.ssnal_en_create(ctypes.byref(ctx), ctypes.byref(bad), None, None) == pkg.EINVAL  # lda < m
    bad = pkg.Matrix(m=3, n=5, lda=3, dtype=0, reserved=0, data=16, col_mean=None, col_scale=None)
    assert L.ssnal_en_create(ctypes.byref(ctx), ctypes.byref(bad), None, None) == pkg.EINVAL  # 24-byte lda
    bad = pkg.Matrix(m=5000, n=5, lda=5000, dtype=0, reserved=0, data=16, col_mean=None, col_scale=None)
    assert L.ssnal_en_create(ctypes.byref(ctx), ctypes.byref(bad), None, None) == pkg.ENOTSUP
    o = pkg.ssnal_en_default_options(mu=0.7)
    ok = pkg.Matrix(m=4, n=5, lda=4, dtype=0, reserved=0, data=16, col_mean=None, col_scale=None)
    assert L.ssnal_en_create(ctypes.byref(ctx), ctypes.byref(ok), ctypes.byref(o), None) == pkg.EINVAL


def test_binding_constants_match_the_header_defines():
    # the binding sizes host buffers from these (a mismatch overruns them)
    import paper_2006_03970_gb300 as pkg
    src = open(os.path.join(ROOT, "include", "ssnal_en.h")).read()
    defines = dict(re.findall(r"#define SSNAL_EN_(\w+)\s+(\d+)", src))
    assert int(defines["PROFILE_PHASES"]) == pkg.PROFILE_PHASES == len(pkg.PHASES)
    assert int(defines["STATIC_MAX_N"]) == pkg.STATIC_MAX_N

"""The C-ABI library builds, loads and exports every entry point declared in
include/xct.h; argument checks that need no GPU reject bad input."""
import ctypes
import os
import re

import pytest

from paper_2009_07226_gb300 import xct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "xct.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(xct_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return xct.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"xct_plan", "xct_project", "xct_backproject", "xct_cgls", "xct_free"} <= set(names)
    raw = ctypes.CDLL(xct.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name


def test_binding_covers_the_header(lib):
    bound = {name for name, _, _ in xct._SIGNATURES}
    assert set(_declared()) == bound


def test_library_is_in_tree(lib):
    assert os.path.dirname(xct.LIB_PATH) == os.path.join(ROOT, "paper_2009_07226_gb300")
    assert xct.xct_version().startswith("xct ")


@pytest.mark.parametrize("kw,msg", [
    (dict(n=0, n_angles=4, n_det=4), "n = 0"),
    (dict(n=40000, n_angles=4, n_det=4), "n = 40000"),
    (dict(n=8, n_angles=0, n_det=4), "n_angles"),
    (dict(n=8, n_angles=4, n_det=-1), "n_angles"),
    (dict(n=8, n_angles=70000, n_det=70000), "2^31"),
    (dict(n=8, n_angles=4, n_det=4, det_spacing=0.0), "det_spacing"),
    (dict(n=8, n_angles=4, n_det=4, det_offset=float("nan")), "det_spacing"),
    (dict(n=8, n_angles=4, n_det=4, min_seg=-1.0), "min_seg"),
    (dict(n=8, n_angles=4, n_det=4, hilbert_tile=-2), "hilbert_tile"),
])
def test_geometry_rejected_before_any_gpu_work(lib, kw, msg):
    g = xct.make_geometry(**kw)
    with pytest.raises(xct.XctError) as e:
        xct.xct_plan(g, "f32")
    assert e.value.status == xct.XCT_ERR_INVALID
    assert msg in str(e.value)


def test_bad_storage_flags_and_table(lib):
    g = xct.make_geometry(8, 4, 4)
    with pytest.raises(xct.XctError):
        xct.xct_plan(g, 7)
    with pytest.raises(xct.XctError):
        xct.xct_plan(g, "f32", flags=0x80)
    import numpy as np
    cs = np.ones((4, 2))
    cs[2, 1] = np.inf
    with pytest.raises(xct.XctError) as e:
        xct.xct_plan(xct.make_geometry(8, 4, 4, cos_sin=cs), "f32")
    assert "angle table" in str(e.value)


def test_null_plan_and_bad_sizes(lib):
    for fn in (lambda: xct.xct_project(None, None, None, 1),
               lambda: xct.xct_backproject(None, None, None, 1),
               lambda: xct.xct_cgls(None, None, None, 1, 3),
               lambda: xct.xct_plan_stats(None)):
        with pytest.raises(xct.XctError) as e:
            fn()
        assert e.value.status == xct.XCT_ERR_INVALID


def test_allocator_callbacks_must_pair(lib):
    r = lib.xct_set_allocator(xct.ALLOC_FN(lambda *a: None), xct.FREE_FN(), None)
    assert r == xct.XCT_ERR_INVALID
    xct.xct_set_allocator(None, None)


def test_binding_constants_match_the_header():
    """Every `#define XCT_...` value of include/xct.h has the same value in
    the Python binding (flags, export selectors, CGLS flags)."""
    with open(os.path.join(ROOT, "include", "xct.h")) as f:
        text = f.read()
    defines = dict(re.findall(r"#define\s+(XCT_[A-Z0-9_]+)\s+(\d+)u?\b", text))
    assert {"XCT_PLAN_PAIRED_ROWS", "XCT_EXPORT_A_PAIRED", "XCT_EXPORT_AT_PAIRED"} <= set(defines)
    for name, value in defines.items():
        assert hasattr(xct, name), name
        assert getattr(xct, name) == int(value), (name, getattr(xct, name), value)


def test_stats_struct_matches_the_header():
    """The binding's xct_stats mirrors the C struct field by field."""
    with open(os.path.join(ROOT, "include", "xct.h")) as f:
        text = f.read()
    end = text.index("} xct_stats;")
    body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for nm in names.split(","):
            fields.append((nm.strip(), ctype))
    size = {"int64_t": 8, "int32_t": 4, "double": 8}
    bound = [(nm, ctypes.sizeof(t)) for nm, t in xct.xct_stats._fields_]
    assert [(nm, size[t]) for nm, t in fields] == bound

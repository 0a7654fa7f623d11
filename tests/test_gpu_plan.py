"""GPU plan vs oracle: the traced matrix, its transpose, the Hilbert
orderings and the packed values, through the C-ABI export calls.

Index structure must be bit-exact; FP64 values within 1e-12 relative (both
sides evaluate the same FP64 expressions without FMA contraction, so in
practice they are identical); stored 16-bit / 32-bit values equal the
oracle's rounding of the FP64 values exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

GEOMS = [
    # n, m, nd, offset, spacing, tile
    (8, 8, 8, 0.0, 1.0, 0),
    (32, 45, 32, 0.13, 1.0, 0),
    (37, 23, 41, -0.4, 0.9, 4),
    (128, 180, 128, 0.0, 1.0, 0),
    (1, 1, 1, 0.0, 1.0, 0),
    (16, 12, 16, 0.0, 1.0, 3),
    (9, 7, 30, 0.5, 1.0, 8),        # many rays miss the grid
    (64, 3, 64, 0.0, 1.0, 16),      # theta = 0, 60, 120 degrees
]


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _oracle(n, m, nd, off, sp):
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off,
                        det_spacing=sp)
    a = oracle.siddon_csr(g)
    return g, a, oracle.transpose(a)


@pytest.mark.parametrize("n,m,nd,off,sp,tile", GEOMS)
def test_matrix_and_transpose_bit_exact(xct, n, m, nd, off, sp, tile):
    g, a, at = _oracle(n, m, nd, off, sp)
    with xct.Plan(n, m, nd, "f32", cos_sin=g.table(), det_offset=off, det_spacing=sp,
                  hilbert_tile=tile, keep_f64=True) as p:
        assert p.stats()["nnz"] == a.nnz
        for what, ref in ((xct.XCT_EXPORT_A_F64, a), (xct.XCT_EXPORT_AT_F64, at)):
            rp, col, val = xct.xct_plan_export(p.handle, what)
            assert np.array_equal(rp, ref.rowptr)
            assert np.array_equal(col, ref.col)
            rel = np.abs(val - ref.val) / np.maximum(np.abs(ref.val), 1e-300)
            assert rel.size == 0 or rel.max() <= 1e-12
            assert np.array_equal(val, ref.val), "values not bit-identical"


@pytest.mark.parametrize("n,m,nd,off,sp,tile", GEOMS[:6])
def test_hilbert_orderings(xct, n, m, nd, off, sp, tile):
    with xct.Plan(n, m, nd, "f32", det_offset=off, det_spacing=sp, hilbert_tile=tile) as p:
        pix, ray = xct.xct_plan_order(p.handle)
    T = tile if tile > 0 else 8
    assert np.array_equal(pix, oracle.hilbert_order(n, n, T, "quad"))
    assert np.array_equal(ray, oracle.hilbert_order(nd, m, T, "col"))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f16a", "bf16a"])
@pytest.mark.parametrize("n,m,nd,off,sp,tile", [GEOMS[1], GEOMS[2], GEOMS[3], GEOMS[6]])
def test_packed_values_are_rounded_matrix(xct, storage, n, m, nd, off, sp, tile):
    g, a, at = _oracle(n, m, nd, off, sp)
    rnd = {"f32": lambda v: v.astype(np.float32).astype(np.float64),
           "f16": lambda v: oracle.round_f16(v * 2.0 ** 15) * 2.0 ** -15,
           "bf16": oracle.round_bf16}[storage.rstrip("a")]
    with xct.Plan(n, m, nd, storage, cos_sin=g.table(), det_offset=off, det_spacing=sp,
                  hilbert_tile=tile) as p:
        for what, ref in ((xct.XCT_EXPORT_A_STORED, a), (xct.XCT_EXPORT_AT_STORED, at)):
            rp, col, val = xct.xct_plan_export(p.handle, what)
            assert np.array_equal(rp, ref.rowptr)
            assert np.array_equal(col, ref.col)
            assert np.array_equal(val, rnd(ref.val))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("n,m,nd,off,sp,tile", GEOMS)
def test_paired_layout_is_rounded_matrix(xct, storage, n, m, nd, off, sp, tile):
    """The paired layouts (XCT_PLAN_PAIRED_ROWS) decoded back: the same
    matrix, every entry once (a shared slot gives one entry to each row of
    its pair), values the oracle's rounding, on every plan geometry
    (ragged Hilbert tiles, rays that miss the grid, a 1-pixel grid)."""
    g, a, at = _oracle(n, m, nd, off, sp)
    rnd = {"f16": lambda v: oracle.round_f16(v * 2.0 ** 15) * 2.0 ** -15, "bf16": oracle.round_bf16}[storage]
    with xct.Plan(n, m, nd, storage, cos_sin=g.table(), det_offset=off, det_spacing=sp,
                  hilbert_tile=tile, paired_rows=True) as p:
        for what, ref in ((xct.XCT_EXPORT_A_PAIRED, a), (xct.XCT_EXPORT_AT_PAIRED, at)):
            rp, col, val = xct.xct_plan_export(p.handle, what)
            assert np.array_equal(rp, ref.rowptr)
            assert np.array_equal(col, ref.col)
            assert np.array_equal(val, rnd(ref.val))


def test_default_angle_table_matches_host_library(xct):
    n, m = 16, 37
    g = oracle.Geometry(n=n, m=m, nd=n)          # oracle default: cos/sin(k*pi/m)
    a = oracle.siddon_csr(g)
    with xct.Plan(n, m, n, "f32", keep_f64=True) as p:
        rp, col, val = xct.xct_plan_export(p.handle, xct.XCT_EXPORT_A_F64)
    assert np.array_equal(rp, a.rowptr) and np.array_equal(col, a.col)
    assert np.array_equal(val, a.val)


def test_plan_stats_are_consistent(xct):
    with xct.Plan(64, 96, 64, "f16") as p:
        st = p.stats()
    assert st["stage_capacity"] > 0 and st["rows_per_block"] == 64
    assert st["slots_a"] >= st["nnz"] and st["slots_at"] >= st["nnz"]
    assert st["bytes_a"] >= 4 * st["nnz"]
    assert st["plan_ms"] > 0


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_autotuned_stage_capacity(xct, storage):
    """XCT_PLAN_AUTOTUNE picks each matrix's stage capacity by timing; the
    layouts stay exact (stored values equal the rounding model) and the
    products agree with the default plan's to the FP32 summation order (a
    row's entries are summed stage by stage, so other stage boundaries
    regroup them)."""
    n, m, nd = 96, 128, 96
    g, a, at = _oracle(n, m, nd, 0.0, 1.0)
    cands = {"f32": (200, 160, 120), "f16": (280, 224, 168)}[storage]
    with xct.Plan(n, m, nd, storage, cos_sin=g.table(), autotune=True) as pt, \
            xct.Plan(n, m, nd, storage, cos_sin=g.table()) as pd:
        st = pt.stats()
        for cap in (st["stage_capacity"], st["stage_capacity_at"]):
            # a candidate, or a candidate reduced until its buffers fit
            assert any(cap <= c and cap % 4 == 0 for c in cands), cap
        rnd = {"f32": lambda v: v.astype(np.float32).astype(np.float64),
               "f16": lambda v: oracle.round_f16(v * 2.0 ** 15) * 2.0 ** -15}[storage]
        for what, ref in ((xct.XCT_EXPORT_A_STORED, a), (xct.XCT_EXPORT_AT_STORED, at)):
            rp, col, val = xct.xct_plan_export(pt.handle, what)
            assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
            assert np.array_equal(val, rnd(ref.val))
        gen = torch.Generator(device="cuda").manual_seed(3)
        x = torch.rand((64, n, n), device="cuda", generator=gen)
        y = torch.rand((64, m, nd), device="cuda", generator=gen)
        for fn in ("project", "backproject"):
            arg = x if fn == "project" else y
            u, v = getattr(pt, fn)(arg), getattr(pd, fn)(arg)
            assert float((u - v).norm() / v.norm()) <= 1e-6, fn

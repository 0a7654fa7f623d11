"""Plans built with XCT_PLAN_NARROW_TILES: the entries of each 4-row group
of the 280-row layouts are reordered (a row's order is free; its FP32 sum
changes only by rounding) so that 16- and 32-slice tiles read staged rows in
distinct bank groups.  Products at every tile width are checked element by
element against the oracle's model of the 16-bit semantics, at the bars of
the product tests, and the stored matrix (export) against the rounded
oracle matrix."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _check(got, want, bound):
    got = np.asarray(got, dtype=np.float64).reshape(want.shape)
    nrm = np.linalg.norm(want)
    if nrm > 0:
        assert np.linalg.norm(got - want) / nrm <= 1e-5
    assert np.all(np.abs(got - want) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("S", [3, 16, 20, 32, 64])
@pytest.mark.parametrize("n,m,nd,off", [(64, 96, 64, 0.0), (37, 23, 41, -0.4)])
def test_narrow_tile_products_vs_oracle_model(xct, kind, S, n, m, nd, off):
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(n + 11 * S)
    mag = 10.0 ** rng.uniform(-3, 3, size=(S, 1))
    x = rng.uniform(-1, 1, size=(S, n * n)) * mag
    y = rng.uniform(-1, 1, size=(S, m * nd)) * mag
    with xct.Plan(n, m, nd, kind, cos_sin=g.table(), det_offset=off, narrow_tiles=True) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, v in ((yo, a, x32), (xo, at, y32)):
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        _check(got.cpu().numpy().reshape(S, -1), oracle.mixed_project(mat, v, kind),
               oracle.project(absm, np.abs(v)))


def test_narrow_tile_export_is_the_rounded_matrix(xct):
    n, m, nd = 48, 64, 48
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table(), narrow_tiles=True) as p:
        for what, ref in ((xct.XCT_EXPORT_A_STORED, a), (xct.XCT_EXPORT_AT_STORED, at)):
            rp, col, val = xct.xct_plan_export(p.handle, what)
            assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
            want = oracle.round_f16(ref.val * 2.0 ** 15) * 2.0 ** -15
            assert np.array_equal(val, want)


def test_flag_needs_a_16bit_matrix(xct):
    with pytest.raises(xct.XctError) as e:
        xct.Plan(32, 20, 32, "f32", narrow_tiles=True)
    assert e.value.status == xct.XCT_ERR_INVALID

"""Plans built with XCT_PLAN_FEW_SLICES: wide-stage layouts of A and A^T
(up to 1524 / 1016 staged 16-byte rows a stage for A / A^T, the packed
entries read straight from device memory) serve products of at most 8
binary16 / bfloat16 slices.
Their products are checked element by element against the oracle's model of
the 16-bit semantics at the bars of the product tests, their CGLS over the
stable phase against the oracle's model of the mixed solve, and a batch that
mixes plans with and without the wide layouts against the plain solves."""
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
@pytest.mark.parametrize("n,m,nd,S,off", [(64, 96, 64, 1, 0.0), (96, 64, 100, 3, 0.25),
                                          (128, 180, 128, 8, 0.0), (37, 23, 41, 5, -0.4),
                                          (128, 180, 128, 9, 0.0)])
def test_wide_products_vs_oracle_model(xct, kind, n, m, nd, S, off):
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(n + 7 * S)
    mag = 10.0 ** rng.uniform(-3, 3, size=(S, 1))
    x = rng.uniform(-1, 1, size=(S, n * n)) * mag
    y = rng.uniform(-1, 1, size=(S, m * nd)) * mag
    with xct.Plan(n, m, nd, kind, cos_sin=g.table(), det_offset=off, few_slices=True) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, v in ((yo, a, x32), (xo, at, y32)):
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        _check(got.cpu().numpy().reshape(S, -1), oracle.mixed_project(mat, v, kind),
               oracle.project(absm, np.abs(v)))


@pytest.mark.parametrize("S", [2, 3, 5])
def test_wide_cgls_stable_phase_vs_oracle_model(xct, S):
    """Two, three or five noisy slices (the 2-, 4- and 8-slice paths of a
    wide tile), k = 1, 3, 5: within 1e-4 of the oracle's model of the
    binary16 solve (the bar of the mixed CGLS test)."""
    import _mixed_envelope as me
    n, m, nd, _, cs, sino, a, at = me.noisy_batch()
    b = sino[:S]
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    b32 = me._to_f32(b.reshape(S, -1))
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, few_slices=True) as p:
        for k in (1, 3, 5):
            xmod, _ = oracle.cgls(*me.mixed_ops(a, at, "f16"), b32, k)
            xg = p.cgls(bt, k).cpu().numpy().reshape(S, -1)
            assert np.linalg.norm(xg - xmod) / np.linalg.norm(xmod) <= 1e-4, k


def test_batch_mixing_wide_and_standard_plans(xct):
    """A batch of jobs on a plan with wide layouts (4 slices) and on one
    without (3 and 20 slices): each job equals its plan's plain solve."""
    n, m, nd = 64, 96, 64
    cs = inputs.angle_table(m)
    rng = np.random.default_rng(3)
    ys = [torch.tensor(rng.uniform(0, 5, size=(S, m, nd)), dtype=torch.float32, device="cuda")
          for S in (4, 3, 20)]
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, few_slices=True) as pw, \
            xct.Plan(n, m, nd, "f16", cos_sin=cs) as ps:
        plans = [pw, ps, ps]
        xs = [torch.empty((y.shape[0], n, n), device="cuda") for y in ys]
        xct.xct_cgls_batch([(p.handle, y, x, y.shape[0]) for p, y, x in zip(plans, ys, xs)], 4)
        for p, y, x in zip(plans, ys, xs):
            ref = p.cgls(y, 4)
            # the batch concatenates jobs of one plan: their slice tile may differ
            # from the job's own, so compare at the stable-phase bar
            assert float((x - ref).norm() / ref.norm()) <= 1e-4


def test_flag_needs_16bit_slices(xct):
    with pytest.raises(xct.XctError) as e:
        xct.Plan(32, 20, 32, "f32", few_slices=True)
    assert e.value.status == xct.XCT_ERR_INVALID

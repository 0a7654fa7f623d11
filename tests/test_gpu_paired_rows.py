"""Plans built with XCT_PLAN_PAIRED_ROWS: paired layouts of A and A^T serve
64-slice tiles of binary16 / bfloat16 slices.  The two rows of a pair share
one staged-row gather for every column both cross; each row's sum is the
same set of products as on the plain layout, in another order (FP32
rounding only).
Checked against the oracle: the decoded paired layout equals the rounded
oracle matrix bit for bit, products element by element against the oracle's
model of the 16-bit semantics at the bars of the product tests, CGLS over the
stable phase against the oracle's model of the mixed solve; and a batch that
mixes plans with and without the paired layouts against the plain solves."""
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
@pytest.mark.parametrize("n,m,nd,off", [(48, 64, 48, 0.0), (37, 23, 41, -0.4), (96, 144, 100, 0.25)])
def test_paired_export_is_the_rounded_matrix(xct, kind, n, m, nd, off):
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    with xct.Plan(n, m, nd, kind, cos_sin=g.table(), det_offset=off, paired_rows=True) as p:
        for what, ref in ((xct.XCT_EXPORT_A_PAIRED, a), (xct.XCT_EXPORT_AT_PAIRED, at)):
            rp, col, val = xct.xct_plan_export(p.handle, what)
            assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
            if kind == "f16":
                want = oracle.round_f16(ref.val * 2.0 ** 15) * 2.0 ** -15
            else:
                want = oracle.round_bf16(ref.val)
            assert np.array_equal(val, want)


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("S", [33, 64, 100, 128])
@pytest.mark.parametrize("n,m,nd,off", [(64, 96, 64, 0.0), (37, 23, 41, -0.4)])
def test_paired_products_vs_oracle_model(xct, kind, S, n, m, nd, off):
    """Slice counts that run as 64-slice tiles (33, 64, 128) and a ragged
    count (100: a 64-slice tile and a partly empty one)."""
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(n + 13 * S)
    mag = 10.0 ** rng.uniform(-3, 3, size=(S, 1))
    x = rng.uniform(-1, 1, size=(S, n * n)) * mag
    y = rng.uniform(-1, 1, size=(S, m * nd)) * mag
    with xct.Plan(n, m, nd, kind, cos_sin=g.table(), det_offset=off, paired_rows=True) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, v in ((yo, a, x32), (xo, at, y32)):
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        _check(got.cpu().numpy().reshape(S, -1), oracle.mixed_project(mat, v, kind),
               oracle.project(absm, np.abs(v)))


def test_paired_products_at_full_tile_on_a_larger_grid(xct):
    """128^2 grid, 192 angles, 128 bins, 64 slices: many stages per block."""
    n, m, nd, S = 128, 192, 128, 64
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, size=(S, n * n))
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table(), paired_rows=True) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
    x32 = x.astype(np.float32).astype(np.float64)
    absm = oracle.CSR(a.nrow, a.ncol, a.rowptr, a.col, np.abs(a.val))
    _check(yo.cpu().numpy().reshape(S, -1), oracle.mixed_project(a, x32, "f16"), oracle.project(absm, x32))


def test_paired_cgls_stable_phase_vs_oracle_model(xct):
    """40 noisy slices (five scaled copies of the 8-slice batch: one 64-slice
    tile), k = 1, 3, 5: within 1e-4 of the oracle's model of the binary16
    solve (the bar of the mixed CGLS test)."""
    import _mixed_envelope as me
    n, m, nd, S0, cs, sino, a, at = me.noisy_batch()
    b = np.concatenate([sino * (1.0 + 0.25 * j) for j in range(5)])
    S = b.shape[0]
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    b32 = me._to_f32(b.reshape(S, -1))
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, paired_rows=True) as p:
        for k in (1, 3, 5):
            xmod, _ = oracle.cgls(*me.mixed_ops(a, at, "f16"), b32, k)
            xg = p.cgls(bt, k).cpu().numpy().reshape(S, -1)
            assert np.linalg.norm(xg - xmod) / np.linalg.norm(xmod) <= 1e-4, k


def test_batch_mixing_paired_and_standard_plans(xct):
    """A batch of jobs on a plan with paired layouts (40 slices) and on one
    without (3 and 50 slices): each job equals its plan's plain solve."""
    n, m, nd = 64, 96, 64
    cs = inputs.angle_table(m)
    rng = np.random.default_rng(4)
    ys = [torch.tensor(rng.uniform(0, 5, size=(S, m, nd)), dtype=torch.float32, device="cuda")
          for S in (40, 3, 50)]
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, paired_rows=True) as pp, \
            xct.Plan(n, m, nd, "f16", cos_sin=cs) as ps:
        plans = [pp, ps, ps]
        xs = [torch.empty((y.shape[0], n, n), device="cuda") for y in ys]
        xct.xct_cgls_batch([(p.handle, y, x, y.shape[0]) for p, y, x in zip(plans, ys, xs)], 4)
        for p, y, x in zip(plans, ys, xs):
            ref = p.cgls(y, 4)
            # the batch concatenates jobs of one plan: their slice tile may differ
            # from the job's own, so compare at the stable-phase bar
            assert float((x - ref).norm() / ref.norm()) <= 1e-4


def test_paired_and_plain_layouts_agree(xct):
    """The same 64 slices on a plan with and one without the paired layouts:
    the same products in another order, within FP32 summation rounding."""
    n, m, nd, S = 64, 96, 64, 64
    cs = inputs.angle_table(m)
    rng = np.random.default_rng(6)
    x = torch.tensor(rng.uniform(0, 1, size=(S, n, n)), dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, paired_rows=True) as pp, \
            xct.Plan(n, m, nd, "f16", cos_sin=cs) as ps:
        y1, y0 = pp.project(x), ps.project(x)
        z1, z0 = pp.backproject(y0), ps.backproject(y0)
    for u, v in ((y1, y0), (z1, z0)):
        assert float((u - v).norm() / v.norm()) <= 1e-6
        assert not torch.equal(u, torch.zeros_like(u))


@pytest.mark.parametrize("kind", ["f32", "f16a", "bf16a"])
def test_flag_needs_16bit_slices(xct, kind):
    with pytest.raises(xct.XctError) as e:
        xct.Plan(32, 20, 32, kind, paired_rows=True)
    assert e.value.status == xct.XCT_ERR_INVALID


def test_paired_export_needs_the_flag(xct):
    with xct.Plan(32, 20, 32, "f16") as p:
        with pytest.raises(xct.XctError) as e:
            xct.xct_plan_export(p.handle, xct.XCT_EXPORT_A_PAIRED)
        assert e.value.status == xct.XCT_ERR_INVALID


def test_paired_stats(xct):
    """Plan statistics of the paired layouts: slots and staged-row reads.
    A pair of rows reads each column it crosses once, so the reads lie
    between half the entries (every column shared) and all of them (none
    shared); neighbouring rays and neighbouring pixels share many."""
    n, m, nd = 64, 96, 64
    with xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m), paired_rows=True) as p, \
            xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m)) as q:
        st, sq = p.stats(), q.stats()
    nnz = st["nnz"]
    for key in ("gathers_a_paired", "gathers_at_paired"):
        assert nnz / 2 <= st[key] < 0.9 * nnz, (key, st[key], nnz)
    assert st["slots_a_paired"] > 0 and st["slots_at_paired"] > 0
    assert sq["slots_a_paired"] == 0 and sq["gathers_a_paired"] == 0
    assert st["slots_a"] == sq["slots_a"] and st["stages_a"] == sq["stages_a"]


@pytest.mark.parametrize("S", [1, 8, 16, 32, 64, 130])
def test_all_layout_flags_together(xct, S):
    """A plan with paired, wide-stage and narrow-tile layouts at once: every
    slice tile runs on its own layout (8-slice tiles on the wide stages,
    16/32 on the reordered 280-row layouts, 64 on the paired ones), each
    product within the bars of the oracle's 16-bit model."""
    n, m, nd = 64, 96, 64
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(100 + S)
    x = rng.uniform(0, 1, size=(S, n * n))
    y = rng.uniform(0, 1, size=(S, m * nd))
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table(), paired_rows=True, few_slices=True,
                  narrow_tiles=True) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, v in ((yo, a, x32), (xo, at, y32)):
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        _check(got.cpu().numpy().reshape(S, -1), oracle.mixed_project(mat, v, "f16"),
               oracle.project(absm, np.abs(v)))


def test_paired_bf16_cgls_stable_phase_vs_oracle_model(xct):
    """bfloat16 storage on paired layouts, 40 noisy slices, k = 1, 3, 5:
    within 5e-4 of the oracle's model of the bfloat16 solve (the bar of the
    mixed CGLS test for bfloat16)."""
    import _mixed_envelope as me
    n, m, nd, S0, cs, sino, a, at = me.noisy_batch()
    b = np.concatenate([sino * (1.0 + 0.25 * j) for j in range(5)])
    S = b.shape[0]
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    b32 = me._to_f32(b.reshape(S, -1))
    with xct.Plan(n, m, nd, "bf16", cos_sin=cs, paired_rows=True) as p:
        for k in (1, 3, 5):
            xmod, _ = oracle.cgls(*me.mixed_ops(a, at, "bf16"), b32, k)
            xg = p.cgls(bt, k).cpu().numpy().reshape(S, -1)
            assert np.linalg.norm(xg - xmod) / np.linalg.norm(xmod) <= 5e-4, k


def test_paired_host_pipeline_equals_device(xct):
    """Host-vector products over three 64-slice tiles (150 slices, the last
    tile ragged) on paired layouts: the pipelined form equals the device
    form bit for bit."""
    n, m, nd, S = 64, 96, 64, 150
    gen = torch.Generator().manual_seed(7)
    x = torch.rand((S, n, n), generator=gen)
    y = torch.rand((S, m, nd), generator=gen)
    with xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m), paired_rows=True) as p:
        yd = p.project(x.cuda()).cpu()
        xd = p.backproject(y.cuda()).cpu()
        xh, yh = x.pin_memory(), y.pin_memory()
        yo = torch.empty((S, m, nd)).pin_memory()
        xo = torch.empty((S, n, n)).pin_memory()
        xct.xct_project(p.handle, xh, yo, S, None)
        xct.xct_backproject(p.handle, yh, xo, S, None)
        torch.cuda.synchronize()
    assert torch.equal(yo, yd) and torch.equal(xo, xd)


def test_paired_resume_is_exact(xct):
    """Checkpoint / resume on paired layouts: 3 iterations, save, 2 more
    from the state equal 5 iterations in one solve bit for bit."""
    import _mixed_envelope as me
    n, m, nd, S0, cs, sino, a, at = me.noisy_batch()
    b = np.concatenate([sino, sino * 1.5, sino * 0.5, sino * 2.0, sino * 0.75])
    S = b.shape[0]
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, paired_rows=True) as p:
        ref = p.cgls(bt, 5)
        state = torch.zeros(xct.xct_cgls_state_bytes(p.handle, S), dtype=torch.uint8, device="cuda")
        x3 = torch.empty((S, n, n), device="cuda")
        xct.xct_cgls_state(p.handle, bt, x3, S, 3, xct.XCT_CGLS_SAVE, state)
        got = torch.empty_like(x3)
        xct.xct_cgls_state(p.handle, None, got, S, 2, xct.XCT_CGLS_RESUME, state)
        torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_paired_products_write_every_output_and_repeat(xct):
    """Poisoned (NaN-filled) outputs are overwritten everywhere, on a ragged
    geometry (rows past the last block, rays that miss the grid), and two
    runs give identical bits (no atomics on the paired path)."""
    n, m, nd, S = 37, 23, 41, 64
    rng = np.random.default_rng(9)
    x = torch.tensor(rng.uniform(0, 1, size=(S, n, n)), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.uniform(0, 1, size=(S, m, nd)), dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m), det_offset=-0.4, paired_rows=True) as p:
        outs = []
        for _ in range(2):
            yo = torch.full((S, m, nd), float("nan"), device="cuda")
            xo = torch.full((S, n, n), float("nan"), device="cuda")
            p.project(x, out=yo)
            p.backproject(y, out=xo)
            torch.cuda.synchronize()
            assert not torch.isnan(yo).any() and not torch.isnan(xo).any()
            outs.append((yo, xo))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_paired_layouts_follow_the_autotuned_capacity(xct):
    """With XCT_PLAN_AUTOTUNE the stage capacity is chosen by timing; the
    paired layouts are built from the chosen layouts and their products
    still meet the bars of the oracle's 16-bit model."""
    n, m, nd, S = 96, 144, 100, 64
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, size=(S, n * n))
    y = rng.uniform(0, 1, size=(S, m * nd))
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table(), paired_rows=True, autotune=True) as p:
        st = p.stats()
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
    assert st["slots_a_paired"] > 0 and st["slots_at_paired"] > 0
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, v in ((yo, a, x32), (xo, at, y32)):
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        _check(got.cpu().numpy().reshape(S, -1), oracle.mixed_project(mat, v, "f16"),
               oracle.project(absm, np.abs(v)))


def test_paired_graph_and_direct_launches_agree(xct):
    """The captured CUDA graph and direct launches of a 40-slice binary16
    solve on paired layouts give the same iterate and residual log bit for
    bit."""
    import _mixed_envelope as me
    n, m, nd, S0, cs, sino, a, at = me.noisy_batch()
    b = np.concatenate([sino * (1.0 + 0.25 * j) for j in range(5)])
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f16", cos_sin=cs, paired_rows=True) as p:
        xg, lg = p.cgls(bt, 8, resid=True)
        xd, ld = p.cgls(bt, 8, resid=True, flags=xct.XCT_CGLS_NO_GRAPH)
    assert torch.equal(xg, xd) and torch.equal(lg, ld)

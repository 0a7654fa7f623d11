"""The matrix-free projection (rays traced again on every call) and back
projection (pixel by pixel, lengths from the pixel's boundary planes)
against the FP64 oracle, against the memoized FP32 products of the same
plan, against each other (adjoint pair), and, for the back projection,
against the stored lengths bit for bit."""
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


@pytest.mark.parametrize("n,m,nd,S,off,sp", [(8, 8, 8, 1, 0.0, 1.0), (37, 23, 41, 5, -0.4, 0.9),
                                             (64, 96, 64, 17, 0.0, 1.0), (9, 7, 30, 3, 0.5, 1.0)])
def test_matfree_projection(xct, n, m, nd, S, off, sp):
    cs = inputs.angle_table(m)
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs, det_offset=off, det_spacing=sp)
    a = oracle.siddon_csr(g)
    rng = np.random.default_rng(n + S)
    x = rng.uniform(-1, 1, size=(S, n * n)).astype(np.float32)
    ref = oracle.project(a, x.astype(np.float64))
    bound = oracle.project(oracle.CSR(a.nrow, a.ncol, a.rowptr, a.col, np.abs(a.val)),
                           np.abs(x.astype(np.float64)))
    with xct.Plan(n, m, nd, "f32", cos_sin=cs, det_offset=off, det_spacing=sp) as p:
        xt = torch.tensor(x.reshape(S, n, n), device="cuda")
        y = torch.full((S, m, nd), float("nan"), device="cuda")
        xct.xct_project_matfree(p.handle, xt, y, S)
        mem = p.project(xt)
        yh = np.zeros((S, m, nd), dtype=np.float32)
        xct.xct_project_matfree(p.handle, x.reshape(S, n, n), yh, S)    # host buffers
    got = y.cpu().numpy().reshape(S, -1).astype(np.float64)
    assert np.array_equal(got, yh.reshape(S, -1))
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)
    if np.linalg.norm(ref) > 0:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        m_np = mem.cpu().numpy().reshape(S, -1).astype(np.float64)
        assert np.linalg.norm(got - m_np) / np.linalg.norm(ref) <= 2e-6


# ---------------------------------------------------------------------------
# matrix-free back projection (pixel by pixel, lengths from the pixel's planes)
# ---------------------------------------------------------------------------

BP_GEOMS = [
    # n, m, nd, S, offset, spacing
    (8, 8, 8, 1, 0.0, 1.0),
    (37, 23, 41, 5, -0.4, 0.9),
    (64, 96, 64, 17, 0.0, 1.0),
    (9, 7, 30, 3, 0.5, 1.0),      # many rays miss the grid
    (16, 4, 16, 2, 0.0, 1.0),     # 0, 45, 90, 135 degrees: rays through corners
    (12, 6, 13, 2, 0.5, 1.0),     # rays along grid lines
]


@pytest.mark.parametrize("n,m,nd,S,off,sp", BP_GEOMS)
def test_matfree_backprojection(xct, n, m, nd, S, off, sp):
    cs = inputs.angle_table(m)
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs, det_offset=off, det_spacing=sp)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(3 * n + S)
    y = rng.uniform(-1, 1, size=(S, m * nd)).astype(np.float32)
    ref = oracle.backproject(at, y.astype(np.float64))
    bound = oracle.backproject(oracle.CSR(at.nrow, at.ncol, at.rowptr, at.col, np.abs(at.val)),
                               np.abs(y.astype(np.float64)))
    with xct.Plan(n, m, nd, "f32", cos_sin=cs, det_offset=off, det_spacing=sp) as p:
        yt = torch.tensor(y.reshape(S, m, nd), device="cuda")
        x = torch.full((S, n, n), float("nan"), device="cuda")
        xct.xct_backproject_matfree(p.handle, yt, x, S)
        mem = p.backproject(yt)
        xh = np.zeros((S, n, n), dtype=np.float32)
        xct.xct_backproject_matfree(p.handle, y.reshape(S, m, nd), xh, S)    # host buffers
        # the transpose of the matrix-free projection
        xr = torch.tensor(rng.uniform(-1, 1, size=(S, n, n)).astype(np.float32), device="cuda")
        yp = torch.empty((S, m, nd), device="cuda")
        xct.xct_project_matfree(p.handle, xr, yp, S)
    got = x.cpu().numpy().reshape(S, -1).astype(np.float64)
    assert np.array_equal(got, xh.reshape(S, -1))
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)
    if np.linalg.norm(ref) > 0:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        m_np = mem.cpu().numpy().reshape(S, -1).astype(np.float64)
        assert np.linalg.norm(got - m_np) / np.linalg.norm(ref) <= 2e-6
    for s in range(S):
        lhs = float(np.dot(yp[s].cpu().numpy().ravel().astype(np.float64), y[s].astype(np.float64)))
        rhs = float(np.dot(xr[s].cpu().numpy().ravel().astype(np.float64), got[s]))
        scale = float(np.dot(np.abs(xr[s].cpu().numpy().ravel()).astype(np.float64),
                             bound[s])) + 1e-30
        assert abs(lhs - rhs) <= 1e-5 * scale


@pytest.mark.parametrize("n,m,nd,off,sp,min_seg", [(16, 4, 16, 0.0, 1.0, 1e-9),
                                                   (12, 6, 13, 0.5, 1.0, 1e-9),
                                                   (9, 7, 30, 0.5, 1.0, 1e-9),
                                                   (10, 9, 11, -0.25, 0.75, 0.0)])
def test_matfree_backprojection_lengths_are_the_stored_values(xct, n, m, nd, off, sp, min_seg):
    """Every ray alone (one slice per ray): the back projection of a unit
    ray is RN32 of its stored lengths, bit for bit, and zero elsewhere.
    With min_seg = 0 the trace also keeps the slivers (below 1e-14) that
    rounding leaves between two crossings that coincide exactly in real
    arithmetic, and the pixel rule does not; they are the only difference."""
    cs = inputs.angle_table(m)
    R = m * nd
    y = np.zeros((R, R), dtype=np.float32)
    np.fill_diagonal(y, 1.0)
    with xct.Plan(n, m, nd, "f32", cos_sin=cs, det_offset=off, det_spacing=sp,
                  min_seg=min_seg) as p:
        rp, col, val = xct.xct_plan_export(p.handle, xct.XCT_EXPORT_A_STORED)
        x = torch.full((R, n, n), float("nan"), device="cuda")
        xct.xct_backproject_matfree(p.handle, torch.tensor(y.reshape(R, m, nd), device="cuda"), x, R)
    x = x.cpu().numpy().reshape(R, -1).astype(np.float64)
    dense = np.zeros((R, n * n))
    for r in range(R):
        # (with min_seg = 0 a zero-length corner segment may repeat a pixel:
        # it adds nothing)
        np.add.at(dense[r], col[rp[r]:rp[r + 1]], val[rp[r]:rp[r + 1]])
    if min_seg > 0:
        assert np.array_equal(x, dense)
    else:
        assert np.abs(x - dense).max() <= 1e-14


# ---------------------------------------------------------------------------
# CGLS without a stored matrix
# ---------------------------------------------------------------------------

def _ops(a, at):
    return (lambda X: oracle.project(a, X)), (lambda Y: oracle.backproject(at, Y))


def test_matfree_cgls_stable_phase(xct):
    """Same recurrence as xct_cgls on the memoized FP32 plan: within the
    FP32 envelope of the FP64 oracle over the stable phase (k <= 5), and
    of the memoized solve."""
    w = inputs.make_workload("cgls2d_128")
    n, m, nd = w["n"], w["m"], w["nd"]
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=w["cos_sin"])
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    b = oracle.project(a, w["images"].reshape(1, -1))
    bt = torch.tensor(b.reshape(1, m, nd), dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f32", cos_sin=g.table()) as p:
        for k in (1, 3, 5):
            x = torch.empty((1, n, n), device="cuda")
            log = torch.zeros((k + 1, 1, 2), dtype=torch.float64, device="cuda")
            xct.xct_cgls_matfree(p.handle, bt, x, 1, k, 0, log)
            xm, lm = p.cgls(bt, k, resid=True)
            xr, lr = oracle.cgls(*_ops(a, at), b, k)
            got = x.cpu().numpy().reshape(1, -1)
            assert np.linalg.norm(got - xr) / np.linalg.norm(xr) <= 2e-5, k
            assert np.linalg.norm(got - xm.cpu().numpy().reshape(1, -1)) / np.linalg.norm(xr) <= 2e-5
            np.testing.assert_allclose(log.cpu().numpy(), lr, rtol=2e-5)


def test_matfree_cgls_x0_stop_and_breakdown(xct):
    n, m, nd, S, k = 24, 30, 26, 3, 3
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(7)
    b = (oracle.project(a, rng.random((S, n * n))) + 0.01 * rng.standard_normal((S, m * nd)))
    b[1] = 0.0
    b = b.astype(np.float32).astype(np.float64)
    x0 = (0.1 * rng.random((S, n * n))).astype(np.float32)
    x0[1] = 0.0
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table()) as p:
        # host buffers, start from x0
        xh = x0.reshape(S, n, n).copy()
        log = np.zeros((k + 1, S, 2))
        xct.xct_cgls_matfree(p.handle, b.astype(np.float32).reshape(S, m, nd), xh, S, k,
                             xct.XCT_CGLS_X0, log)
        xr, lr = oracle.cgls(*_ops(a, at), b, k, x0=x0.astype(np.float64))
        got = xh.reshape(S, -1).astype(np.float64)
        assert np.array_equal(got[1], x0[1])
        for s in (0, 2):
            assert np.linalg.norm(got[s] - xr[s]) / np.linalg.norm(xr[s]) <= 2e-5
        np.testing.assert_allclose(log[:, [0, 2]], lr[:, [0, 2]], rtol=2e-5)
        # zero data: every slice stops at k = 0
        with pytest.raises(xct.XctError) as e:
            xz = torch.full((2, n, n), 5.0, device="cuda")
            xct.xct_cgls_matfree(p.handle, torch.zeros((2, m, nd), device="cuda"), xz, 2, 2)
        assert e.value.status == xct.XCT_ERR_BREAKDOWN
        assert torch.count_nonzero(xz) == 0

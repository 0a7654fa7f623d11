"""The matrix-free projection (rays traced again on every call) against the
FP64 oracle and against the memoized FP32 projection of the same plan."""
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

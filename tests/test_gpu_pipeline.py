"""Host-buffer products over several slice tiles run as a pipeline: each
tile's host-to-device copy, pack, product, unpack and device-to-host copy,
with the copies on a second stream overlapping the neighbouring tiles'
products.  Every tile is computed as in the one-launch device form, so the
results must be identical bit for bit; pinned and pageable host memory,
and one host side with the other on the device.  The pipelined products
are also checked element by element against the oracle (its FP64 products
for FP32 storage, its model of the 16-bit semantics otherwise) at the bars
of the product tests: relative L2 <= 1e-5 and each output within 1e-5 of
the sum of |a_e v_e| over its row."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND = 64, 96, 64


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.mark.parametrize("storage,S", [("f16", 150), ("bf16", 65), ("f32", 70), ("f16a", 40),
                                       ("f16", 64)])
def test_host_pipeline_equals_device(xct, storage, S):
    g = torch.Generator().manual_seed(S)
    x = torch.rand((S, N, N), generator=g) - 0.3
    y = torch.rand((S, M, ND), generator=g)
    with xct.Plan(N, M, ND, storage, cos_sin=inputs.angle_table(M)) as p:
        yd = p.project(x.cuda()).cpu()
        xd = p.backproject(y.cuda()).cpu()
        # pinned host buffers
        xh, yh = x.pin_memory(), torch.empty((S, M, ND)).pin_memory()
        xct.xct_project(p.handle, xh, yh, S)
        assert torch.equal(yh, yd)
        xo = torch.empty((S, N, N)).pin_memory()
        xct.xct_backproject(p.handle, y.pin_memory(), xo, S)
        assert torch.equal(xo, xd)
        # pageable host buffers
        yn = np.empty((S, M, ND), np.float32)
        xct.xct_project(p.handle, x.numpy(), yn, S)
        assert np.array_equal(yn, yd.numpy())
        # device input, host output; host input, device output
        yh2 = torch.empty((S, M, ND)).pin_memory()
        xct.xct_project(p.handle, x.cuda(), yh2, S)
        assert torch.equal(yh2, yd)
        yd2 = torch.empty((S, M, ND), device="cuda")
        xct.xct_project(p.handle, xh, yd2, S)
        assert torch.equal(yd2.cpu(), yd)
    # the pipelined results against the oracle
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=inputs.angle_table(M))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    x64 = x.numpy().reshape(S, -1).astype(np.float64)
    y64 = y.numpy().reshape(S, -1).astype(np.float64)
    for got, mat, v in ((yh, a, x64), (xo, at, y64)):
        if storage in ("f16", "bf16"):
            want = oracle.mixed_project(mat, v, storage)
        elif storage in ("f16a", "bf16a"):
            want = oracle.matrix16_project(mat, v, storage[:-1])
        else:
            want = oracle.project(mat, v)
        absm = oracle.CSR(mat.nrow, mat.ncol, mat.rowptr, mat.col, np.abs(mat.val))
        bound = oracle.project(absm, np.abs(v))
        got = got.numpy().reshape(S, -1).astype(np.float64)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5
        assert np.all(np.abs(got - want) <= 1e-5 * bound + 1e-30)

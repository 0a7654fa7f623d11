"""xct_project_noalloc: the projection for callers that cannot allocate
device memory during a call (device memory owned up front by another
component, or a latency-critical loop).  Its working memory is the library's
fixed 32 MiB device array, shared by all calls; these checks compare it with
xct_project on consecutive calls (so stale contents of the shared array would
show) and check the size and pointer limits.  Collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("kind,S", [("f32", 5), ("f32", 40), ("f16", 17), ("f16", 64), ("bf16", 33)])
def test_matches_xct_project_on_consecutive_calls(xct, kind, S):
    n, m, nd = 96, 72, 100
    gen = torch.Generator(device="cuda").manual_seed(S)
    with xct.Plan(n, m, nd, kind, det_offset=0.25) as p:
        for call in range(2):
            # a different magnitude per call: stale maxima or staging data from
            # the previous call would change the result
            x = torch.rand((S, n, n), device="cuda", generator=gen) * (10.0 ** (2 * call - 1))
            y_ref = p.project(x)
            y = torch.full((S, m, nd), float("nan"), device="cuda")
            xct.xct_project_noalloc(p.handle, x, y, S)
            torch.cuda.synchronize()
            assert torch.isfinite(y).all()
            assert _rel(y, y_ref) <= 1e-5
            assert torch.allclose(y, y_ref, rtol=1e-5, atol=1e-6 * float(y_ref.abs().max()))


def test_rejects_sizes_beyond_the_fixed_array(xct):
    with xct.Plan(512, 64, 512, "f32") as p:
        S = 64     # 64 * (512^2 + 64 * 512) * 4 bytes > 32 MiB
        x = torch.zeros((S, 512, 512), device="cuda")
        y = torch.zeros((S, 64, 512), device="cuda")
        with pytest.raises(xct.XctError) as e:
            xct.xct_project_noalloc(p.handle, x, y, S)
        assert e.value.status == xct.XCT_ERR_INVALID
        assert "fixed array" in str(e.value)
        xct.xct_project_noalloc(p.handle, x[:2], y[:2], 2)   # a small call still works


def test_rejects_host_buffers(xct):
    with xct.Plan(32, 20, 32, "f32") as p:
        x = np.zeros((1, 32, 32), dtype=np.float32)
        y = np.zeros((1, 20, 32), dtype=np.float32)
        with pytest.raises(xct.XctError) as e:
            xct.xct_project_noalloc(p.handle, x, y, 1)
        assert "device pointers" in str(e.value)

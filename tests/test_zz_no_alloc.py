"""xct_project_noalloc: the projection for callers that cannot allocate
device memory during a call (device memory owned up front by another
component, or a latency-critical loop).  Its working memory is the library's
fixed 32 MiB device array, shared by all calls; these checks compare it with
xct_project on consecutive calls (so stale contents of the shared array would
show), check that a call allocates nothing (no allocator callback, no change
in the device's free memory, even on the first call after the plan was
built) and check the size and pointer limits.  Collected last on purpose."""
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


class _CountingAllocator:
    """Routes the library's allocations through PyTorch's caching allocator
    and counts them."""

    def __init__(self):
        self.calls = 0

    def alloc(self, nbytes, stream):
        self.calls += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  stream if stream else 0)

    def release(self, ptr, nbytes, stream):
        self.calls += 1
        torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("kind,S,paired", [("f32", 5, False), ("f32", 40, False), ("f16", 17, False),
                                            ("f16", 64, False), ("bf16", 33, False), ("f16", 64, True)])
def test_matches_xct_project_on_consecutive_calls(xct, kind, S, paired):
    """Also on a plan with paired layouts, whose 64-slice tiles run the
    paired kernel in both calls."""
    n, m, nd = 96, 72, 100
    gen = torch.Generator(device="cuda").manual_seed(S)
    with xct.Plan(n, m, nd, kind, det_offset=0.25, paired_rows=paired) as p:
        for call in range(2):
            # a different magnitude per call: stale maxima or staging data from
            # the previous call would change the result
            x = torch.rand((S, n, n), device="cuda", generator=gen) * (10.0 ** (2 * call - 1))
            y_ref = p.project(x)
            y = torch.full((S, m, nd), float("nan"), device="cuda")
            torch.cuda.synchronize()
            counter = _CountingAllocator()
            xct.xct_set_allocator(counter.alloc, counter.release)
            try:
                free0 = torch.cuda.mem_get_info()[0]
                xct.xct_project_noalloc(p.handle, x, y, S)
                torch.cuda.synchronize()
                free1 = torch.cuda.mem_get_info()[0]
            finally:
                xct.xct_set_allocator(None, None)
            assert counter.calls == 0
            # the fixed array became resident when the plan was built, so not
            # even the first call changes the device's free memory
            assert free1 == free0
            # the same kernels on the same tiles as xct_project
            assert torch.equal(y, y_ref)


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


def test_the_documented_bound_is_exact(xct):
    """The header's working-memory formula at its edge: 64 binary16 slices
    of a 256^2 grid with 256 bins need 6*64*256^2 + 4*64*M*256 bytes for the
    vectors plus 512 for the maxima and the work counter.  With M = 128 that
    is 512 bytes more than 32 MiB (rejected), with M = 127 it fits."""
    n, nd, S = 256, 256, 64

    def need(m):
        r = lambda b: (b + 255) // 256 * 256
        return r(4 * S * n * n) + r(4 * S * m * nd) + r(2 * S * n * n) + r(4 * S) + 256

    assert need(127) <= 32 << 20 < need(128) == (32 << 20) + 512
    x = torch.rand((S, n, n), device="cuda")
    with xct.Plan(n, 127, nd, "f16") as p:
        y = torch.empty((S, 127, nd), device="cuda")
        xct.xct_project_noalloc(p.handle, x, y, S)
        torch.cuda.synchronize()
        assert torch.equal(y, p.project(x))
    with xct.Plan(n, 128, nd, "f16") as p:
        y = torch.empty((S, 128, nd), device="cuda")
        with pytest.raises(xct.XctError) as e:
            xct.xct_project_noalloc(p.handle, x, y, S)
        assert e.value.status == xct.XCT_ERR_INVALID
        xct.xct_project_noalloc(p.handle, x[:32], y[:32], 32)   # half of it fits


def test_rejects_host_buffers(xct):
    with xct.Plan(32, 20, 32, "f32") as p:
        x = np.zeros((1, 32, 32), dtype=np.float32)
        y = np.zeros((1, 20, 32), dtype=np.float32)
        with pytest.raises(xct.XctError) as e:
            xct.xct_project_noalloc(p.handle, x, y, 1)
        assert "device pointers" in str(e.value)

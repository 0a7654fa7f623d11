"""Failure paths on the GPU without a GPU fault: the bounded waits of the
persistent product kernel run out (limit set to 0), the kernel gives up
cleanly, the plan reports XCT_ERR_TIMEOUT, and the context stays usable;
device allocations fail at a chosen point (injected through the allocator
callbacks) and every call returns XCT_ERR_OOM with nothing leaked."""
import numpy as np
import pytest
import torch

from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND, S = 96, 128, 96, 64     # 64 binary16 slices: the persistent kernel


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _data():
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand((S, N, N), device="cuda", generator=g)
    y = torch.rand((S, M, ND), device="cuda", generator=g)
    return x, y


@pytest.mark.parametrize("paired", [False, True])
def test_wait_limit_zero_times_out_and_recovers(xct, paired):
    """On the plain layouts and on paired ones (the same waits in the
    paired kernel)."""
    x, y = _data()
    with xct.Plan(N, M, ND, "f16", cos_sin=inputs.angle_table(M), paired_rows=paired) as p:
        ref = p.project(x).clone()
        torch.cuda.synchronize()
        xct.xct_plan_check(p.handle)
        prev = xct.xct_set_wait_limit(0)
        try:
            outcomes = []
            for _ in range(3):
                yo = torch.full_like(ref, float("nan"))
                xct.xct_project(p.handle, x, yo, S)
                try:
                    xct.xct_plan_check(p.handle)
                    outcomes.append("ok")
                except xct.XctError as e:
                    assert e.status == xct.XCT_ERR_TIMEOUT
                    outcomes.append("timeout")
            with pytest.raises(xct.XctError) as ei:
                for _ in range(3):
                    p.cgls(y, 3)
            assert ei.value.status == xct.XCT_ERR_TIMEOUT
        finally:
            assert xct.xct_set_wait_limit(prev) == 0
        assert "timeout" in outcomes, outcomes
        # the context and the plan are usable again, results unchanged
        torch.cuda.synchronize()
        xct.xct_plan_check(p.handle)
        again = p.project(x)
        torch.cuda.synchronize()
        xct.xct_plan_check(p.handle)
        assert torch.equal(again, ref)
        x4 = p.cgls(y, 3)
        assert torch.isfinite(x4).all()


def test_wait_limit_validation(xct):
    with pytest.raises(xct.XctError) as ei:
        xct.xct_set_wait_limit(61_000_000_000)
    assert ei.value.status == xct.XCT_ERR_INVALID
    assert xct.xct_set_wait_limit(2_000_000_000) == 2_000_000_000


class _Budget:
    """Allocator callbacks that serve `ok` allocations, then fail (None:
    never fail; count only)."""

    def __init__(self, ok=None):
        self.ok = ok
        self.live = {}
        self.count = 0

    def alloc(self, nbytes, stream):
        self.count += 1
        if self.ok is not None and self.count > self.ok:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                 stream if stream else 0)
        self.live[ptr] = nbytes
        return ptr

    def release(self, ptr, nbytes, stream):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def _plan_and_solve(xct, geom, y, flags=0):
    h = xct.xct_plan(geom, "f16", flags)
    try:
        xo = torch.empty((S, N, N), device="cuda")
        xct.xct_cgls(h, y, xo, S, 3)
        torch.cuda.synchronize()
    finally:
        xct.xct_free(h)


@pytest.mark.parametrize("paired", [False, True])
def test_allocation_failures_return_oom_without_leaks(xct, paired):
    """Also for a plan with paired layouts (their build is the last part of
    the plan's, so the failure points near the end fall inside it)."""
    flags = xct.XCT_PLAN_PAIRED_ROWS if paired else 0
    cs = inputs.angle_table(M)
    geom = xct.make_geometry(N, M, ND, cs)
    _, y = _data()
    # count the allocations of one plan build and one solve
    counter = _Budget()
    xct.xct_set_allocator(counter.alloc, counter.release)
    try:
        h = xct.xct_plan(geom, "f16", flags)
        n_plan = counter.count
        xct.xct_free(h)
        _plan_and_solve(xct, geom, y, flags)
        n_total = counter.count - n_plan
    finally:
        xct.xct_set_allocator(None, None)
    torch.cuda.synchronize()
    assert counter.live == {} and n_total > n_plan > 5
    for ok in (0, 1, n_plan // 2, n_plan - 12, n_plan - 5, n_plan - 1, n_plan + 2, n_total - 1):
        budget = _Budget(ok)
        xct.xct_set_allocator(budget.alloc, budget.release)
        try:
            with pytest.raises(xct.XctError) as ei:
                _plan_and_solve(xct, geom, y, flags)
            assert ei.value.status == xct.XCT_ERR_OOM, (ok, str(ei.value))
            assert "allocator callback failed" in str(ei.value)
        finally:
            xct.xct_set_allocator(None, None)
        torch.cuda.synchronize()
        assert budget.live == {}, f"{len(budget.live)} allocations leaked (budget {ok})"
    # the default allocator serves the same calls again
    _plan_and_solve(xct, geom, y, flags)

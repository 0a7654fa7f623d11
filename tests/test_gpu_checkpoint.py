"""Exact CGLS checkpoint and resume (xct_cgls_state): k iterations with the
state saved, then m iterations resumed from it, give the x and residual log
of k + m uninterrupted iterations bit for bit -- from device or host state
buffers, in FP32 and binary16 storage, with or without a CUDA graph; a state
of another plan or slice count is rejected."""
import numpy as np
import pytest
import torch

from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND, S = 64, 96, 64, 5


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def sino():
    cs = inputs.angle_table(M)
    ells = inputs.random_ellipsoids(np.random.default_rng(9), 20)
    out = np.stack([inputs.line_integrals(inputs.cut_ellipsoids(ells, inputs.slice_z(s, S)), N, cs, ND)
                    for s in range(S)])
    for s in range(S):
        out[s] = inputs.poisson_noise(np.random.default_rng(300 + s), out[s], N, 1e4)
    return torch.tensor(out, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("host_state", [False, True])
@pytest.mark.parametrize("flags", [0, 2])            # graph / XCT_CGLS_NO_GRAPH
def test_save_then_resume_is_exact(xct, sino, storage, host_state, flags):
    with xct.Plan(N, M, ND, storage, cos_sin=inputs.angle_table(M)) as p:
        x10, log10 = p.cgls(sino, 10, resid=True, flags=flags)
        nbytes = xct.xct_cgls_state_bytes(p.handle, S)
        assert nbytes > 4 * S * (2 * N * N + M * ND)
        state = (np.zeros(nbytes, dtype=np.uint8) if host_state
                 else torch.zeros(nbytes, dtype=torch.uint8, device="cuda"))
        x4 = torch.empty((S, N, N), device="cuda")
        log4 = torch.zeros((5, S, 2), dtype=torch.float64, device="cuda")
        xct.xct_cgls_state(p.handle, sino, x4, S, 4, flags | xct.XCT_CGLS_SAVE, state, log4)
        assert torch.equal(x4, p.cgls(sino, 4, flags=flags))
        assert torch.equal(log4, log10[:5])
        # continue 3 and save again, then 3 more
        x7 = torch.empty_like(x4)
        log7 = torch.zeros((4, S, 2), dtype=torch.float64, device="cuda")
        xct.xct_cgls_state(p.handle, None, x7, S, 3, flags | xct.XCT_CGLS_RESUME | xct.XCT_CGLS_SAVE,
                           state, log7)
        x10b = torch.empty_like(x4)
        log10b = torch.zeros((4, S, 2), dtype=torch.float64, device="cuda")
        xct.xct_cgls_state(p.handle, None, x10b, S, 3, flags | xct.XCT_CGLS_RESUME, state, log10b)
        torch.cuda.synchronize()
    assert torch.equal(log7, log10[4:8])
    assert torch.equal(x10b, x10)
    assert torch.equal(log10b, log10[7:])


def test_state_of_another_problem_is_rejected(xct, sino):
    with xct.Plan(N, M, ND, "f32", cos_sin=inputs.angle_table(M)) as p, \
            xct.Plan(N, M + 4, ND, "f32", cos_sin=inputs.angle_table(M + 4)) as q:
        state = torch.zeros(xct.xct_cgls_state_bytes(p.handle, S), dtype=torch.uint8, device="cuda")
        x = torch.empty((S, N, N), device="cuda")
        with pytest.raises(xct.XctError) as e0:       # nothing saved yet
            xct.xct_cgls_state(p.handle, None, x, S, 2, xct.XCT_CGLS_RESUME, state)
        assert e0.value.status == xct.XCT_ERR_INVALID
        xct.xct_cgls_state(p.handle, sino, x, S, 2, xct.XCT_CGLS_SAVE, state)
        y2 = torch.zeros((S, M + 4, ND), device="cuda")
        big = torch.zeros(xct.xct_cgls_state_bytes(q.handle, S), dtype=torch.uint8, device="cuda")
        big[:state.numel()] = state
        with pytest.raises(xct.XctError) as e1:       # another geometry
            xct.xct_cgls_state(q.handle, y2, x, S, 2, xct.XCT_CGLS_RESUME, big)
        assert e1.value.status == xct.XCT_ERR_INVALID
        with pytest.raises(xct.XctError) as e2:       # neither flag
            xct.xct_cgls_state(p.handle, sino, x, S, 2, 0, state)
        assert e2.value.status == xct.XCT_ERR_INVALID

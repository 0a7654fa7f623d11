"""Exact CGLS checkpoint and resume (xct_cgls_state): k iterations with the
state saved, then m iterations resumed from it, give the x and residual log
of k + m uninterrupted iterations bit for bit -- from device or host state
buffers, in FP32 and binary16 storage, with or without a CUDA graph; a state
of another plan or slice count is rejected.  Over the stable phase (k + m
<= 5 iterations) a resumed solve also equals the oracle's: the FP64 CGLS
within 2e-5 (FP32 storage, the bar of the plain solver) and the oracle's
model of the binary16 solve within 1e-4 (the bar of the mixed solver)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND, S = 64, 96, 64, 5


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _sino_host():
    cs = inputs.angle_table(M)
    ells = inputs.random_ellipsoids(np.random.default_rng(9), 20)
    out = np.stack([inputs.line_integrals(inputs.cut_ellipsoids(ells, inputs.slice_z(s, S)), N, cs, ND)
                    for s in range(S)])
    for s in range(S):
        out[s] = inputs.poisson_noise(np.random.default_rng(300 + s), out[s], N, 1e4)
    return out.astype(np.float32)


@pytest.fixture(scope="module")
def sino():
    return torch.tensor(_sino_host(), device="cuda")


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


@pytest.mark.parametrize("storage,k,m", [("f32", 2, 3), ("f32", 4, 1), ("f16", 2, 3)])
def test_resumed_stable_phase_equals_the_oracle(xct, sino, storage, k, m):
    """k iterations saved, m resumed (k + m <= 5, the stable phase): the
    iterate and the residual log against the oracle's solve of k + m
    iterations on the same FP32 sinogram."""
    import _mixed_envelope as me
    b = _sino_host().reshape(S, -1).astype(np.float64)
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=inputs.angle_table(M))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    if storage == "f32":
        ops, tol = ((lambda X: oracle.project(a, X)), (lambda Y: oracle.backproject(at, Y))), 2e-5
    else:
        ops, tol = me.mixed_ops(a, at, storage), 1e-4
    xr, lr = oracle.cgls(*ops, b, k + m)
    with xct.Plan(N, M, ND, storage, cos_sin=inputs.angle_table(M)) as p:
        state = torch.zeros(xct.xct_cgls_state_bytes(p.handle, S), dtype=torch.uint8, device="cuda")
        x = torch.empty((S, N, N), device="cuda")
        log1 = torch.zeros((k + 1, S, 2), dtype=torch.float64, device="cuda")
        xct.xct_cgls_state(p.handle, sino, x, S, k, xct.XCT_CGLS_SAVE, state, log1)
        log2 = torch.zeros((m + 1, S, 2), dtype=torch.float64, device="cuda")
        xct.xct_cgls_state(p.handle, None, x, S, m, xct.XCT_CGLS_RESUME, state, log2)
        torch.cuda.synchronize()
    xg = x.cpu().numpy().reshape(S, -1)
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= tol
    log = np.concatenate([log1.cpu().numpy(), log2.cpu().numpy()[1:]])
    np.testing.assert_allclose(log[:, :, 0], lr[:, :, 0], rtol=tol)
    # ||A^T r_k|| is the norm of A^T b - A^T A x_k: a relative error in
    # either term is amplified by ||A^T b|| / ||A^T r_k||
    amp = float(np.max(lr[0, :, 1] / lr[:, :, 1]))
    np.testing.assert_allclose(log[:, :, 1], lr[:, :, 1], rtol=tol * amp)

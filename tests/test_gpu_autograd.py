"""Differentiable projector, TV kernel, Adam kernel and the regularised
reconstruction (Eq. 1 with R = lam * TV_eps) on the GPU.

FP32 storage: the TV value within 1e-6 and its gradient within 1e-5 (relative
L2) of the FP64 oracle; the gradient of the whole cost through the autograd
Functions within 1e-5 of the oracle's analytic FP64 gradient (itself pinned by
finite differences in tests/test_oracle_tv_loss.py); the Adam kernel within
1e-6 of PyTorch's FP32 Adam."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND, S = 32, 45, 32, 2
LAM, EPS = 1e-3, 1e-3


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def small():
    cs = inputs.angle_table(M)
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=cs)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(21)
    y = rng.uniform(0, 5, size=(S, M * ND)).astype(np.float32)
    x = rng.uniform(0, 1, size=(S, N * N)).astype(np.float32)
    return cs, a, at, x, y


def test_tv_kernel_vs_oracle(xct):
    rng = np.random.default_rng(3)
    for n, s in ((1, 1), (7, 2), (33, 3), (128, 2)):
        x = rng.uniform(0, 1, size=(s, n, n)).astype(np.float32)
        x[:, : n // 2] = 0.5                       # flat regions: |dx| << eps
        val_ref, g_ref = oracle.tv_value_grad(x.astype(np.float64), EPS)
        xt = torch.tensor(x, device="cuda")
        grad = torch.empty_like(xt)
        val = np.zeros(s)
        xct.xct_tv(xt, n, s, EPS, 2.0, grad, val)
        assert abs(val.sum() - 2.0 * val_ref) <= 1e-6 * 2.0 * val_ref
        g = grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - 2.0 * g_ref) <= 1e-5 * np.linalg.norm(2.0 * g_ref) + 1e-12


def test_adam_kernel_vs_torch(xct):
    torch.manual_seed(0)
    p0 = torch.randn(10007, device="cuda")
    grads = [torch.randn(10007, device="cuda") for _ in range(5)]
    ref = p0.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=1e-2, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    x = p0.clone()
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    for t, g in enumerate(grads, start=1):
        opt.zero_grad()
        ref.grad = g.clone()
        opt.step()
        xct.xct_adam(x, g, m, v, x.numel(), 1e-2, 0.9, 0.999, 1e-8, t)
    torch.cuda.synchronize()
    assert float((x - ref.detach()).norm() / (ref.detach() - p0).norm()) <= 1e-5


def test_autograd_projector_is_the_adjoint_pair(xct):
    from paper_2009_07226_gb300 import autograd as ag
    with xct.Plan(48, 40, 50, "f32", det_offset=0.2) as p:
        x = torch.rand((3, 48, 48), device="cuda", requires_grad=True)
        w = torch.rand((3, 40, 50), device="cuda")
        (ag.project(x, p) * w).sum().backward()
        assert torch.equal(x.grad, p.backproject(w))
        yv = torch.rand((3, 40, 50), device="cuda", requires_grad=True)
        u = torch.rand((3, 48, 48), device="cuda")
        (ag.backproject(yv, p) * u).sum().backward()
        assert torch.equal(yv.grad, p.project(u))
        lhs = (p.project(x.detach()).double() * w.double()).sum()
        rhs = (x.detach().double() * p.backproject(w).double()).sum()
        assert abs(float(lhs - rhs)) <= 1e-6 * abs(float(lhs))


def test_cost_gradient_vs_oracle(xct, small):
    from paper_2009_07226_gb300 import autograd as ag
    cs, a, at, x, y = small
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    r = oracle.project(a, x64) - y64
    ref = oracle.backproject(at, r) + LAM * oracle.tv_value_grad(x64.reshape(S, N, N), EPS)[1].reshape(S, -1)
    with xct.Plan(N, M, ND, "f32", cos_sin=cs) as p:
        xt = torch.tensor(x.reshape(S, N, N), device="cuda", requires_grad=True)
        yt = torch.tensor(y.reshape(S, M, ND), device="cuda")
        res = ag.project(xt, p) - yt
        loss = 0.5 * (res * res).sum() + ag.tv(xt, EPS, LAM)
        loss.backward()
    g = xt.grad.cpu().numpy().reshape(S, -1).astype(np.float64)
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)
    want = 0.5 * float((r * r).sum()) + LAM * oracle.tv_value_grad(x64.reshape(S, N, N), EPS)[0]
    assert abs(float(loss.detach()) - want) <= 1e-5 * want


def test_datafit_function_vs_oracle(xct, small):
    """The data term through library calls only (projection, xct_datafit,
    back projection): value 0.5 ||A x - y||^2 and gradient A^T (A x - y)
    against the FP64 oracle, with an incoming gradient of 3."""
    from paper_2009_07226_gb300 import autograd as ag
    cs, a, at, x, y = small
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    r = oracle.project(a, x64) - y64
    with xct.Plan(N, M, ND, "f32", cos_sin=cs) as p:
        xt = torch.tensor(x.reshape(S, N, N), device="cuda", requires_grad=True)
        yt = torch.tensor(y.reshape(S, M, ND), device="cuda")
        val = ag.datafit(xt, yt, p)
        (3.0 * val).backward()
        # value also through a host pointer
        q = p.project(xt.detach())
        rr = torch.empty_like(q)
        host = np.zeros(1)
        xct.xct_datafit(q, yt, rr, M * ND, S, host)
    want = 0.5 * float((r * r).sum())
    assert abs(float(val) - want) <= 1e-5 * want
    assert abs(host[0] - float(val)) == 0.0
    np.testing.assert_allclose(rr.cpu().numpy().reshape(S, -1), r, rtol=0, atol=1e-5 * np.abs(r).max())
    g = xt.grad.cpu().numpy().reshape(S, -1).astype(np.float64)
    ref = 3.0 * oracle.backproject(at, r)
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)


def test_native_reconstruction_matches_autograd_loop(xct, small):
    from paper_2009_07226_gb300 import autograd as ag
    cs, a, at, x, y = small
    steps = 3
    with xct.Plan(N, M, ND, "f32", cos_sin=cs) as p:
        yt = torch.tensor(y.reshape(S, M, ND), device="cuda")
        xa, la = ag.tv_reconstruct(p, yt, steps=steps, lr=1e-2, lam=LAM, eps=EPS, history=True)
        xn = torch.empty((S, N, N), device="cuda")
        ln = np.zeros(steps)
        xct.xct_tv_reconstruct(p.handle, yt, xn, S, steps, 1e-2, LAM, EPS, 0, ln)
    np.testing.assert_allclose(ln, la, rtol=1e-5)
    # the cost at the start (x = 0) is 0.5 ||y||^2 + lam * n^2 * eps per slice
    want0 = 0.5 * float((y.astype(np.float64) ** 2).sum()) + LAM * S * N * N * EPS
    assert abs(ln[0] - want0) <= 1e-6 * want0
    assert float((xn - xa).norm() / xa.norm()) <= 1e-4


@pytest.mark.parametrize("kind,tol", [("f32", 1e-5), ("bf16", 1e-2)])
def test_native_reconstruction_vs_oracle(xct, kind, tol):
    """60 Adam steps on a 3-slice ellipsoid phantom: the cost history against
    the FP64 oracle's Adam reconstruction of the same cost."""
    n, m, nd, s, steps, lr = 64, 96, 64, 3, 60, 1e-2
    cs = inputs.angle_table(m)
    ells = inputs.random_ellipsoids(np.random.default_rng(4), 20)
    sino = np.stack([inputs.line_integrals(inputs.cut_ellipsoids(ells, inputs.slice_z(k, s)), n, cs, nd)
                     for k in range(s)]).astype(np.float32)
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs)
    a = oracle.siddon_csr(g)
    xr, hr = oracle.adam_tv_reconstruct(a, oracle.transpose(a), sino.reshape(s, -1), n, steps, lr, LAM, EPS)
    with xct.Plan(n, m, nd, kind, cos_sin=cs) as p:
        x = torch.empty((s, n, n), device="cuda")
        loss = np.zeros(steps)
        xct.xct_tv_reconstruct(p.handle, torch.tensor(sino, device="cuda"), x, s, steps, lr, LAM, EPS, 0, loss)
    dl = float(np.max(np.abs(loss - hr) / hr))
    dx = float(np.linalg.norm(x.cpu().numpy().reshape(s, -1) - xr) / np.linalg.norm(xr))
    print(f"{kind}: max relative cost deviation {dl:.3e}, relative x deviation {dx:.3e}")
    assert np.all(np.isfinite(loss)) and torch.isfinite(x).all()
    assert hr[-1] < 0.1 * hr[0]
    assert dl <= tol
    assert dx <= 10 * tol

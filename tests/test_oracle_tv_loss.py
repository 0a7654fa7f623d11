"""Pin of the oracle's regularised cost (Eq. 1 with R = lam * TV_eps): the
analytic gradient A^T (A x - y) + lam grad TV_eps equals FP64 central finite
differences of 0.5 ||A x - y||^2 + lam TV_eps(x) on the 32 x 32, 45-angle,
32-bin, 2-slice instance."""
import numpy as np
import torch

import oracle
from paper_2009_07226_gb300 import inputs


def test_loss_gradient_by_central_differences():
    n, m, nd, S = 32, 45, 32, 2
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(21)
    y = rng.uniform(0, 5, size=(S, m * nd))
    x = rng.uniform(0, 1, size=(S, n * n))
    lam, eps = 1e-3, 1e-3

    def loss(xv):
        r = oracle.project(a, xv) - y
        return 0.5 * float((r * r).sum()) + lam * oracle.tv_value_grad(xv.reshape(S, n, n), eps)[0]

    r = oracle.project(a, x) - y
    grad = oracle.backproject(at, r) + lam * oracle.tv_value_grad(x.reshape(S, n, n), eps)[1].reshape(S, -1)
    h = 1e-6
    idx = rng.choice(S * n * n, 60, replace=False)
    fd = np.empty(idx.size)
    for q, k in enumerate(idx):
        xp = x.copy().reshape(-1)
        xm = x.copy().reshape(-1)
        xp[k] += h
        xm[k] -= h
        fd[q] = (loss(xp.reshape(S, -1)) - loss(xm.reshape(S, -1))) / (2 * h)
    ref = grad.reshape(-1)[idx]
    assert np.linalg.norm(fd - ref) <= 1e-6 * np.linalg.norm(ref)


def test_adam_reconstruction_equals_torch_adam():
    n, m, nd, S = 24, 30, 26, 2
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m))
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(5)
    y = rng.uniform(0, 3, size=(S, m * nd))
    lam, eps, lr, steps = 2e-2, 1e-2, 5e-2, 12
    x, hist = oracle.adam_tv_reconstruct(a, at, y, n, steps, lr, lam, eps)
    # the same cost as a torch graph: dense A (a library matmul), TV written
    # with torch ops, gradient by autograd, update by torch.optim.Adam
    dense = torch.zeros((m * nd, n * n), dtype=torch.float64)
    for row in range(m * nd):
        lo, hi = a.rowptr[row], a.rowptr[row + 1]
        dense[row, torch.from_numpy(a.col[lo:hi].astype(np.int64))] = torch.from_numpy(a.val[lo:hi])
    xt = torch.zeros((S, n * n), dtype=torch.float64, requires_grad=True)
    yt = torch.from_numpy(y)
    opt = torch.optim.Adam([xt], lr=lr, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    ref = []
    for _ in range(steps):
        opt.zero_grad()
        xi = xt.view(S, n, n)
        dx = torch.nn.functional.pad(xi[:, :, 1:] - xi[:, :, :-1], (0, 1))
        dy = torch.nn.functional.pad(xi[:, 1:, :] - xi[:, :-1, :], (0, 0, 0, 1))
        r = xt @ dense.T - yt
        cost = 0.5 * (r * r).sum() + lam * torch.sqrt(dx * dx + dy * dy + eps * eps).sum()
        ref.append(float(cost))
        cost.backward()
        opt.step()
    np.testing.assert_allclose(hist, ref, rtol=1e-12)
    assert np.abs(x - xt.detach().numpy()).max() <= 1e-9
    assert hist[-1] < hist[0]

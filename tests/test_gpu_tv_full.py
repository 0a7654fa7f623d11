"""The regularised reconstruction at full size (1024^2 grid, 720 angles,
1024 bins, 16 slices, BF16 storage, lam 1e-3, eps 1e-3, lr 1e-2), where the
FP64 oracle cannot run 200 steps.  Checked instead: the cost at x = 0 in
closed form; the first Adam step at sampled pixels, which from x = 0 is
-lr * g / (|g| + 1e-8) with g = -A^T y computed by the oracle pixel by
pixel; and after 200 steps, the cost the fused loop reports for the final
iterate against the same cost assembled from separate projection and TV
calls."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = inputs.WORKLOADS["tv3d_1024"]
N, M, ND, S, STEPS = W["n"], W["m"], W["nd"], W["slices"], W["iters"]
LAM, EPS, LR = 1e-3, 1e-3, 1e-2


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def work():
    w = inputs.make_workload("tv3d_1024", with_images=False)
    return w, w["sino"].astype(np.float32)


def test_first_step_and_initial_cost(xct, work):
    w, y = work
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=w["cos_sin"])
    rng = np.random.default_rng(41)
    pick = [3, 12]
    pixels = np.sort(rng.choice(N * N, 24, replace=False))
    ref_g = -oracle.backproject_pixels(g, y.reshape(S, -1)[pick].astype(np.float64), pixels)
    with xct.Plan(N, M, ND, "bf16", cos_sin=w["cos_sin"]) as p:
        x = torch.empty((S, N, N), device="cuda")
        loss = np.zeros(1)
        xct.xct_tv_reconstruct(p.handle, torch.tensor(y, device="cuda"), x, S, 1, LR, LAM, EPS, 0, loss)
        got = x.reshape(S, -1)[pick][:, torch.tensor(pixels, device="cuda")].double().cpu().numpy()
    want0 = 0.5 * float((y.astype(np.float64) ** 2).sum()) + LAM * S * N * N * EPS
    assert abs(loss[0] - want0) <= 1e-6 * want0
    big = np.abs(ref_g) > 1e-3 * np.abs(ref_g).max()
    assert big.sum() >= 10
    np.testing.assert_allclose(got[big], -LR * np.sign(ref_g[big]), rtol=1e-6)
    assert np.all(np.abs(got[~big]) <= LR * (1 + 1e-6))


def test_full_run_cost_consistency(xct, work):
    w, y = work
    with xct.Plan(N, M, ND, "bf16", cos_sin=w["cos_sin"]) as p:
        yt = torch.tensor(y, device="cuda")
        x = torch.empty((S, N, N), device="cuda")
        loss = np.zeros(STEPS)
        xct.xct_tv_reconstruct(p.handle, yt, x, S, STEPS, LR, LAM, EPS, 0, loss)
        # cost of the final iterate: one more step started from it reports
        # the cost before its update
        xf = x.clone()
        last = np.zeros(1)
        xct.xct_tv_reconstruct(p.handle, yt, x, S, 1, LR, LAM, EPS, 1, last)
        r = p.project(xf) - yt
        tv = np.zeros(S)
        xct.xct_tv(xf, N, S, EPS, LAM, None, tv)
        torch.cuda.synchronize()
        sep = 0.5 * float((r.double() ** 2).sum()) + float(tv.sum())
    print(f"cost: start {loss[0]:.6e}, step 200 {loss[-1]:.6e}, final {last[0]:.6e}")
    assert np.all(np.isfinite(loss)) and np.isfinite(last[0])
    assert loss[-1] < 0.1 * loss[0]
    assert abs(last[0] - sep) <= 1e-6 * sep

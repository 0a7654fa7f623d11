"""Parity on the large geometry (1536^2 grid, 1024 angles, 1536 bins,
A with about 3.4e9 entries, 32 slices), where the FP64 oracle cannot hold A:
it computes sampled outputs one by one, matrix-free (projections of sampled
rays, back projections of sampled pixels), and for two of the slices the
true residual ||y - A x|| of the 30-iteration mixed-precision CGLS iterate,
which must equal the residual the solver logged."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = inputs.WORKLOADS["large3d_1536"]
N, M, ND, S = W["n"], W["m"], W["nd"], W["slices"]


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def geom():
    return oracle.Geometry(n=N, m=M, nd=ND, cos_sin=inputs.angle_table(M))


@pytest.fixture(scope="module")
def sampled(geom):
    rng = np.random.default_rng(31)
    x = rng.uniform(0, 1, size=(S, N * N)).astype(np.float32)
    y = rng.uniform(0, 1, size=(S, M * ND)).astype(np.float32)
    rays = np.sort(rng.choice(M * ND, 256, replace=False))
    pixels = np.sort(rng.choice(N * N, 32, replace=False))
    pick = [S // 4, 3 * S // 4]
    ref_y = oracle.project_rays(geom, x[pick].astype(np.float64), rays)
    ref_x = oracle.backproject_pixels(geom, y[pick].astype(np.float64), pixels)
    return x, y, rays, pixels, pick, ref_y, ref_x


@pytest.mark.parametrize("kind", ["f32", "f16"])
def test_products_sampled(xct, geom, sampled, kind):
    x, y, rays, pixels, pick, ref_y, ref_x = sampled
    with xct.Plan(N, M, ND, kind, cos_sin=geom.table()) as p:
        assert p.stats()["nnz"] > 2_800_000_000
        yo = p.project(torch.tensor(x.reshape(S, N, N), device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, M, ND), device="cuda"))
        torch.cuda.synchronize()
        gy = yo.reshape(S, -1)[pick][:, torch.tensor(rays, device="cuda")].double().cpu().numpy()
        gx = xo.reshape(S, -1)[pick][:, torch.tensor(pixels, device="cuda")].double().cpu().numpy()
        del yo, xo
    tol = 1e-5 if kind == "f32" else 2.0 ** -11
    for got, ref in ((gy, ref_y), (gx, ref_x)):
        for s in range(len(pick)):
            assert np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s]) <= tol, kind


def test_mixed_cgls_residual_of_two_slices(xct, geom):
    w = inputs.make_workload("large3d_1536", with_images=False)
    K = w["iters"]
    b = w["sino"].astype(np.float32)
    # two slices through the middle of the phantom (the end slices of the
    # volume may cut no ellipsoid and have an all-zero sinogram)
    pick = [S // 4, 3 * S // 4]
    assert np.all(np.linalg.norm(b.reshape(S, -1)[pick], axis=1) > 0)
    with xct.Plan(N, M, ND, "f16", cos_sin=w["cos_sin"]) as p:
        xk, log = p.cgls(torch.tensor(b, device="cuda"), K, resid=True)
        torch.cuda.synchronize()
        xs = xk.reshape(S, -1)[pick].double().cpu().numpy()
        lg = log.cpu().numpy()
        del xk
    r0 = lg[0, pick, 0]
    rk = lg[-1, pick, 0]
    # CGLS residual norms decrease monotonically (slack for rounding)
    assert np.all(np.diff(lg[:, pick, 0], axis=0) <= 1e-6 * r0)
    assert np.all(rk < 0.5 * r0)
    bb = b.reshape(S, -1)[pick].astype(np.float64)
    true_r = np.linalg.norm(bb - oracle.project_rays(geom, xs), axis=1)
    # the logged residual is updated with the 16-bit product; the oracle
    # recomputes it with the FP64 matrix
    assert np.all(np.abs(rk - true_r) <= 1e-2 * true_r), (rk, true_r)
    assert np.allclose(r0, np.linalg.norm(bb, axis=1), rtol=1e-6)


@pytest.fixture(scope="module")
def two_slices(geom):
    """The FP64 oracle's CGLS of two slices, 3 iterations, matrix-free."""
    w = inputs.make_workload("large3d_1536", with_images=False)
    b = w["sino"].astype(np.float32)
    pick = [S // 4, 3 * S // 4]
    bp = b.reshape(S, -1)[pick].astype(np.float64)
    xr, lr = oracle.cgls(lambda X: oracle.project_rays(geom, X),
                         lambda Y: oracle.backproject_rays(geom, Y), bp, 3)
    return w, b, pick, xr, lr


@pytest.mark.parametrize("kind,tol", [("f32", 2e-5), ("f16", 2e-3)])
def test_cgls_stable_phase_of_two_slices_vs_oracle(xct, two_slices, kind, tol):
    """The 32-slice solve of the large workload against the FP64 oracle's
    CGLS of two of its slices over the stable phase (3 iterations), the
    oracle's products computed matrix-free (A of this size does not fit in
    host memory): the iterate after 3 iterations and the residual log
    (||r_k||, ||A^T r_k||, k = 0..3) within the stable-phase bars of the
    plain solver (FP32: 2e-5; binary16: 2e-3, as on the 3D batch).  The
    two slices cut the phantom through its middle (an end slice of the
    volume may cut no ellipsoid)."""
    w, b, pick, xr, lr = two_slices
    with xct.Plan(N, M, ND, kind, cos_sin=w["cos_sin"]) as p:
        xk, log = p.cgls(torch.tensor(b, device="cuda"), 3, resid=True)
        torch.cuda.synchronize()
        xs = xk.reshape(S, -1)[pick].double().cpu().numpy()
        lg = log.cpu().numpy()[:, pick, :]
        del xk
    for s in range(2):
        assert np.linalg.norm(xs[s] - xr[s]) / np.linalg.norm(xr[s]) <= tol, (kind, s)
    np.testing.assert_allclose(lg, lr, rtol=tol)

"""Parity at the benchmark's full size (512^2 grid, 768 angles, 512 bins,
64 slices) in the launch configuration the benchmark times (slice tiles of
64 for 16-bit storage, 32 for FP32; the benchmark's binary16 solve on paired
layouts, XCT_PLAN_PAIRED_ROWS).  The oracle computes sampled outputs
one by one: projections of sampled rays and back projections of sampled
pixels (matrix-free), and the full FP64 CGLS of two sampled slices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

N, M, ND, S = 512, 768, 512, 64


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def setup():
    cs = inputs.angle_table(M)
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=cs)
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, size=(S, N * N)).astype(np.float32)
    y = rng.uniform(0, 1, size=(S, M * ND)).astype(np.float32)
    rays = np.sort(rng.choice(M * ND, 384, replace=False))
    pixels = np.sort(rng.choice(N * N, 96, replace=False))
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    ref_y = oracle.project_rays(g, x64, rays)          # [S, 384]
    ref_x = oracle.backproject_pixels(g, y64, pixels)  # [S, 96]
    return g, x, y, rays, pixels, ref_y, ref_x


@pytest.mark.parametrize("kind", ["f32", "f16", "bf16", "f16-paired", "bf16-paired"])
def test_products_sampled(xct, setup, kind):
    g, x, y, rays, pixels, ref_y, ref_x = setup
    kind, paired = kind.split("-")[0], kind.endswith("-paired")
    with xct.Plan(N, M, ND, kind, cos_sin=g.table(), paired_rows=paired) as p:
        yo = p.project(torch.tensor(x.reshape(S, N, N), device="cuda"))
        xo = p.backproject(torch.tensor(y.reshape(S, M, ND), device="cuda"))
        torch.cuda.synchronize()
    gy = yo.reshape(S, -1)[:, torch.tensor(rays, device="cuda")].double().cpu().numpy()
    gx = xo.reshape(S, -1)[:, torch.tensor(pixels, device="cuda")].double().cpu().numpy()
    if kind == "f32":
        # lengths are positive and inputs non-negative: |a x| sums = the outputs
        for got, ref in ((gy, ref_y), (gx, ref_x)):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
            assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-30)
    else:
        u = 2.0 ** -11 if kind == "f16" else 2.0 ** -8
        for got, ref in ((gy, ref_y), (gx, ref_x)):
            for s in range(S):
                assert np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s]) < u


@pytest.mark.slow
def test_cgls_sampled_slices(xct):
    """The benchmark's CGLS (64 noisy slices): slices 0 and 63 of the
    batched GPU solve against the FP64 oracle's solve of those slices alone
    (slices are independent problems), over the stable phase (4
    iterations); over the full 50 iterations, the logged residual of each
    sampled slice equals the residual of the returned iterate."""
    w = inputs.make_workload("batch3d_512", with_images=False)
    K = w["iters"]
    g = oracle.Geometry(n=N, m=M, nd=ND, cos_sin=w["cos_sin"])
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    pick = [0, S - 1]
    b = w["sino"].reshape(S, -1)
    xo, logo = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y),
                           b[pick], 4)
    bt = torch.tensor(w["sino"], dtype=torch.float32, device="cuda")
    for kind, tol in (("f32", 2e-5), ("f16", 2e-3), ("f16-paired", 2e-3)):
        storage, paired = kind.split("-")[0], kind.endswith("-paired")
        with xct.Plan(N, M, ND, storage, cos_sin=w["cos_sin"], paired_rows=paired) as p:
            x4 = p.cgls(bt, 4).reshape(S, -1)[pick].double().cpu().numpy()
            xk, log = p.cgls(bt, K, resid=True)
        assert np.linalg.norm(x4 - xo) / np.linalg.norm(xo) <= tol, kind
        xk = xk.reshape(S, -1)[pick].double().cpu().numpy()
        true_r = np.linalg.norm(b[pick] - oracle.project(a, xk), axis=1)
        got_r = log.cpu().numpy()[-1, pick, 0]
        # f32: drift of the updated residual; f16: the residual is updated
        # with the 16-bit product, the recomputation uses the FP64 matrix
        rtol = 1e-3 if storage == "f32" else 1e-2
        assert np.all(np.abs(got_r - true_r) <= rtol * true_r), (kind, got_r, true_r)


def test_fp64_products_sampled(xct, setup):
    """The double-precision form at full size: sampled rays and pixels
    against the oracle within the FP64 summation bound (inputs and lengths
    are non-negative, so sum |a x| is the output itself): 2 gamma_n with n
    up to 2 * 512 * 1.5 terms per output, under 4e-13 relative."""
    g, x, y, rays, pixels, ref_y, ref_x = setup
    with xct.Plan(N, M, ND, "f16", cos_sin=g.table(), keep_f64=True) as p:
        yo = p.project_f64(torch.tensor(x.reshape(S, N, N), dtype=torch.float64, device="cuda"))
        xo = p.backproject_f64(torch.tensor(y.reshape(S, M, ND), dtype=torch.float64,
                                            device="cuda"))
        torch.cuda.synchronize()
    gy = yo.reshape(S, -1)[:, torch.tensor(rays, device="cuda")].cpu().numpy()
    gx = xo.reshape(S, -1)[:, torch.tensor(pixels, device="cuda")].cpu().numpy()
    for got, ref in ((gy, ref_y), (gx, ref_x)):
        assert np.all(np.abs(got - ref) <= 4e-13 * ref + 1e-300)

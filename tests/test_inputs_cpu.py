"""The seeded input generators: reproducible, the closed-form line integrals
equal independent computations, the noise models have the stated
statistics, and the workload recipes have the stated shapes."""
import math

import numpy as np

from paper_2009_07226_gb300 import inputs


def test_workloads_are_reproducible():
    a = inputs.make_workload("small3d_64")
    b = inputs.make_workload("small3d_64")
    assert np.array_equal(a["sino"], b["sino"]) and np.array_equal(a["images"], b["images"])
    assert a["sino"].shape == (4, 96, 64) and a["images"].shape == (4, 64, 64)


def test_disk_line_integrals_are_chords():
    """A centred disk of radius r (pixels) and density rho: every line at
    offset t has integral 2 rho sqrt(r^2 - t^2), whatever the angle."""
    n, m, nd = 64, 7, 64
    ells = np.array([[0.0, 0.0, 0.5, 0.5, 0.3, 1.7]])      # radius 0.5 * n/2 = 16 px
    cs = inputs.angle_table(m)
    li = inputs.line_integrals(ells, n, cs, nd, spacing=0.75, offset=0.1)
    t = (np.arange(nd) - 0.5 * (nd - 1)) * 0.75 + 0.1
    ref = 2 * 1.7 * np.sqrt(np.maximum(16.0 ** 2 - t ** 2, 0.0))
    assert np.allclose(li, ref[None, :], rtol=1e-12, atol=1e-12)


def test_ellipse_line_integrals_match_quadrature():
    """A rotated off-centre ellipse: the closed form against midpoint
    quadrature of its indicator along each line."""
    n = 64
    ells = np.array([[0.2, -0.1, 0.35, 0.15, 0.7, 0.9]])
    cs = inputs.angle_table(5)
    nd = 9
    li = inputs.line_integrals(ells, n, cs, nd, spacing=3.0)
    cx, cy, a, b, phi, rho = ells[0]
    h = n / 2
    s = np.linspace(-n, n, 400001)
    ds = s[1] - s[0]
    for k in range(cs.shape[0]):
        c, sn = cs[k]
        for j in range(nd):
            t = (j - 0.5 * (nd - 1)) * 3.0
            px, py = t * c - s * sn, t * sn + s * c        # points of the line, pixel units
            dx, dy = px / h - cx, py / h - cy
            xr = dx * math.cos(phi) + dy * math.sin(phi)
            yr = -dx * math.sin(phi) + dy * math.cos(phi)
            inside = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
            assert abs(rho * inside.sum() * ds - li[k, j]) <= 2e-3 * max(1.0, li[k, j])


def test_ellipsoid_cuts():
    ells = np.array([[0.1, 0.2, 0.0, 0.3, 0.2, 0.5, 0.4, 1.0]])
    cut = inputs.cut_ellipsoids(ells, 0.3)               # z = 0.3 of a c = 0.5 ellipsoid
    f = math.sqrt(1 - (0.3 / 0.5) ** 2)
    assert np.allclose(cut, [[0.1, 0.2, 0.3 * f, 0.2 * f, 0.4, 1.0]])
    assert inputs.cut_ellipsoids(ells, 0.6).shape == (0, 6)
    assert [inputs.slice_z(s, 4) for s in range(4)] == [-0.75, -0.25, 0.25, 0.75]


def test_poisson_noise_statistics():
    """At I0 photons, -log(counts / I0) scaled back to pixel units is
    unbiased to first order with variance (n/2)^2 exp(p) / I0."""
    n, i0 = 64, 1e4
    sino = np.full((200, 500), 20.0)                    # p = 2 * 20 / 64 = 0.625
    noisy = inputs.poisson_noise(np.random.default_rng(3), sino, n, i0)
    p = 2 * 20.0 / n
    assert abs(noisy.mean() - 20.0) < 0.05
    var = (n / 2) ** 2 * math.exp(p) / i0
    assert abs(noisy.var() / var - 1) < 0.05


def test_batch_jobs_recipe():
    jobs = inputs.batch_jobs()
    assert len(jobs) == 64
    assert {j["n"] for j in jobs} <= {256, 384, 512, 768}
    assert all(j["m"] == 3 * j["n"] // 2 and j["nd"] == j["n"] for j in jobs)
    assert all(1 <= j["slices"] <= 32 for j in jobs)
    assert len({j["seed"] for j in jobs}) == 64
    assert jobs == inputs.batch_jobs()

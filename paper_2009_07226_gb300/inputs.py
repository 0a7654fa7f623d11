"""Seeded synthetic inputs for the parallel-beam workloads.

This module generates data only: angle lists, random ellipse / ellipsoid
phantoms, their exact continuous line integrals (a closed form of the Radon
transform of an ellipse, independent of any discretisation) and measurement
noise.  It holds none of the reconstruction method's arithmetic (no Siddon
trace, no system matrix, no solver) and is the only module that both the
CUDA path's tests and the CPU oracle use.

Conventions (shared with the library and the oracle):
  * the grid has n x n unit pixels centred at the origin; pixel (ix, iy) has
    its centre at (ix - n/2 + 1/2, iy - n/2 + 1/2); phantoms are defined in
    normalised coordinates u = 2 * position / n, so the unit disk fills the
    grid;
  * ray (k, j) is the line {P : P . (cos th_k, sin th_k) = t_j} with
    t_j = (j - (nd - 1)/2) * spacing + offset.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Workloads (sizes of the benchmark configurations)
# ---------------------------------------------------------------------------

WORKLOADS = {
    # plain 2D CGLS, one slice
    "cgls2d_128": dict(n=128, m=180, nd=128, slices=1, iters=30, seed=1,
                       phantom="ellipses", count=10, rho=(-0.3, 1.0), noise=None),
    # batched 3D, plain vs mixed precision
    "batch3d_512": dict(n=512, m=768, nd=512, slices=64, iters=50, seed=2,
                        phantom="ellipsoids", count=20, rho=(0.0, 1.0),
                        noise=("poisson", 1e4)),
    # large mixed precision
    "large3d_1536": dict(n=1536, m=1024, nd=1536, slices=32, iters=30, seed=3,
                         phantom="ellipsoids", count=20, rho=(0.0, 1.0),
                         noise=("gaussian", 0.05)),
    # differentiable, TV-regularised
    "tv3d_1024": dict(n=1024, m=720, nd=1024, slices=16, iters=200, seed=4,
                      phantom="ellipsoids", count=20, rho=(0.0, 1.0), noise=None),
    # small 3D volume (slice-sharding checks on the host)
    "small3d_64": dict(n=64, m=96, nd=64, slices=4, iters=10, seed=5,
                       phantom="ellipsoids", count=20, rho=(0.0, 1.0),
                       noise=("poisson", 1e4)),
}


def angle_table(m: int) -> np.ndarray:
    """[m, 2] float64 (cos th_k, sin th_k), th_k = k * pi / m, from the C
    library's cos/sin (Python's math module)."""
    cs = np.empty((m, 2), dtype=np.float64)
    for k in range(m):
        th = k * math.pi / m
        cs[k, 0] = math.cos(th)
        cs[k, 1] = math.sin(th)
    return cs


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

def random_ellipses(rng: np.random.Generator, count: int, rho=(-0.3, 1.0)) -> np.ndarray:
    """[count, 6] rows (cx, cy, a, b, phi, rho) in normalised coordinates:
    centres uniform in the unit disk (radius sqrt(U), angle 2 pi U),
    semi-axes U[0.05, 0.4], rotation U[0, pi), density U[rho]."""
    out = np.empty((count, 6))
    for i in range(count):
        r = math.sqrt(rng.uniform())
        a = 2.0 * math.pi * rng.uniform()
        out[i, 0] = r * math.cos(a)
        out[i, 1] = r * math.sin(a)
        out[i, 2] = rng.uniform(0.05, 0.4)
        out[i, 3] = rng.uniform(0.05, 0.4)
        out[i, 4] = rng.uniform(0.0, math.pi)
        out[i, 5] = rng.uniform(rho[0], rho[1])
    return out


def random_ellipsoids(rng: np.random.Generator, count: int, rho=(0.0, 1.0)) -> np.ndarray:
    """[count, 8] rows (cx, cy, cz, a, b, c, phi, rho): (cx, cy) uniform in
    the unit disk, cz U[-0.8, 0.8], semi-axes U[0.05, 0.4], rotation phi
    U[0, pi) about the rotation (z) axis only, density U[rho]."""
    out = np.empty((count, 8))
    for i in range(count):
        r = math.sqrt(rng.uniform())
        a = 2.0 * math.pi * rng.uniform()
        out[i, 0] = r * math.cos(a)
        out[i, 1] = r * math.sin(a)
        out[i, 2] = rng.uniform(-0.8, 0.8)
        out[i, 3] = rng.uniform(0.05, 0.4)
        out[i, 4] = rng.uniform(0.05, 0.4)
        out[i, 5] = rng.uniform(0.05, 0.4)
        out[i, 6] = rng.uniform(0.0, math.pi)
        out[i, 7] = rng.uniform(rho[0], rho[1])
    return out


def slice_z(s: int, slices: int) -> float:
    """Height of slice s: the slices span the phantom, z_s = -1 + (2s+1)/S."""
    return -1.0 + (2.0 * s + 1.0) / slices


def cut_ellipsoids(ells: np.ndarray, z: float) -> np.ndarray:
    """2D ellipses (cx, cy, a, b, phi, rho) where the plane at height z cuts
    the ellipsoids: semi-axes scale by sqrt(1 - ((z - cz)/c)^2)."""
    rows = []
    for cx, cy, cz, a, b, c, phi, rho in ells:
        u = (z - cz) / c
        if abs(u) < 1.0:
            f = math.sqrt(1.0 - u * u)
            rows.append((cx, cy, a * f, b * f, phi, rho))
    return np.array(rows, dtype=np.float64).reshape(-1, 6)


def rasterize(ells: np.ndarray, n: int) -> np.ndarray:
    """[n, n] image, row iy / column ix: sum of densities of the ellipses
    containing each pixel centre."""
    c = (np.arange(n) - n / 2 + 0.5) * (2.0 / n)
    ux, uy = np.meshgrid(c, c)            # ux varies along columns (ix)
    img = np.zeros((n, n))
    for cx, cy, a, b, phi, rho in ells:
        dx, dy = ux - cx, uy - cy
        xr = dx * math.cos(phi) + dy * math.sin(phi)
        yr = -dx * math.sin(phi) + dy * math.cos(phi)
        img += rho * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img


def line_integrals(ells: np.ndarray, n: int, cos_sin: np.ndarray, nd: int,
                   spacing: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """[m, nd] exact line integrals of the continuous ellipse phantom, in
    pixel units.  For an ellipse with semi-axes A, B (pixel units), rotation
    phi, centre (X0, Y0) and density rho, the line P . (cos th, sin th) = t
    has chord 2 A B sqrt(sigma^2 - tau^2) / sigma^2 when tau^2 <= sigma^2,
    with sigma^2 = A^2 cos^2(th - phi) + B^2 sin^2(th - phi) and
    tau = t - (X0 cos th + Y0 sin th)."""
    cs = np.asarray(cos_sin, dtype=np.float64).reshape(-1, 2)
    t = (np.arange(nd) - 0.5 * (nd - 1)) * spacing + offset
    out = np.zeros((cs.shape[0], nd))
    h = n / 2.0
    for cx, cy, a, b, phi, rho in ells:
        A, B, X0, Y0 = a * h, b * h, cx * h, cy * h
        cphi, sphi = math.cos(phi), math.sin(phi)
        # cos(th - phi), sin(th - phi) from the table
        cd = cs[:, 0] * cphi + cs[:, 1] * sphi
        sd = cs[:, 1] * cphi - cs[:, 0] * sphi
        sig2 = (A * cd) ** 2 + (B * sd) ** 2
        tau = t[None, :] - (X0 * cs[:, 0] + Y0 * cs[:, 1])[:, None]
        rad = sig2[:, None] - tau * tau
        out += np.where(rad > 0, 2.0 * rho * A * B * np.sqrt(np.maximum(rad, 0.0)) / sig2[:, None], 0.0)
    return out


# ---------------------------------------------------------------------------
# Noise
# ---------------------------------------------------------------------------

def poisson_noise(rng: np.random.Generator, sino: np.ndarray, n: int, i0: float) -> np.ndarray:
    """Photon-count noise: line integrals in field-of-view units p = (2/n) y,
    counts ~ Poisson(i0 exp(-p)) clamped to >= 1, returned as
    (n/2) * (-log(counts / i0))."""
    p = sino * (2.0 / n)
    counts = rng.poisson(i0 * np.exp(-p)).astype(np.float64)
    counts = np.maximum(counts, 1.0)
    return (n / 2.0) * (-np.log(counts / i0))


def gaussian_noise(rng: np.random.Generator, sino: np.ndarray, frac: float) -> np.ndarray:
    """Additive white noise with sigma = frac * RMS of the slice's sinogram."""
    rms = math.sqrt(float(np.mean(sino * sino))) if sino.size else 0.0
    return sino + rng.normal(0.0, frac * rms, size=sino.shape)


# ---------------------------------------------------------------------------
# Whole workloads
# ---------------------------------------------------------------------------

def make_workload(name: str, slices: int | None = None, slice_offset: int = 0,
                  with_images: bool = True, volume_slices: int | None = None,
                  noiseless: bool = False):
    """Phantom volume [S, n, n] (or None) and measured sinograms [S, m, nd]
    (float64) for one of WORKLOADS, seeded by the workload's seed.  Slices
    [slice_offset, slice_offset + slices) of a volume of `volume_slices`
    slices (default: the workload's slice count) are produced, so ranks
    sharing a volume get disjoint slice ranges of the same phantom.  With
    noiseless=True the sinograms are the exact line integrals (no noise
    drawn)."""
    w = WORKLOADS[name]
    n, m, nd = w["n"], w["m"], w["nd"]
    total = w["slices"] if volume_slices is None else volume_slices
    S = total if slices is None else slices
    cs = angle_table(m)
    rng = np.random.default_rng(w["seed"])
    if w["phantom"] == "ellipses":
        ells2 = random_ellipses(rng, w["count"], w["rho"])
        cuts = [ells2] * S
    else:
        ells3 = random_ellipsoids(rng, w["count"], w["rho"])
        cuts = [cut_ellipsoids(ells3, slice_z(slice_offset + s, total)) for s in range(S)]
    imgs = np.stack([rasterize(c, n) for c in cuts]) if with_images else None
    sino = np.stack([line_integrals(c, n, cs, nd) for c in cuts]) if S else np.zeros((0, m, nd))
    noise = w["noise"]
    for s in range(S):
        nrng = np.random.default_rng(1_000_000 * w["seed"] + slice_offset + s)
        if noise is None or noiseless:
            continue
        if noise[0] == "poisson":
            sino[s] = poisson_noise(nrng, sino[s], n, noise[1])
        elif noise[0] == "gaussian":
            sino[s] = gaussian_noise(nrng, sino[s], noise[1])
    return dict(n=n, m=m, nd=nd, slices=S, iters=w["iters"], cos_sin=cs,
                images=imgs, sino=sino)


# ---------------------------------------------------------------------------
# Uneven batch of reconstruction jobs
# ---------------------------------------------------------------------------

BATCH = dict(count=64, sizes=(256, 384, 512, 768), max_slices=32, iters=20, seed=6,
             ellipses=10, photons=1e4)


def batch_jobs(count: int = BATCH["count"], seed: int = BATCH["seed"],
               sizes=BATCH["sizes"], max_slices: int = BATCH["max_slices"]) -> list:
    """Seeded job list of the uneven batch: grid side N drawn uniformly from
    `sizes`, M = 1.5 N angles on [0, pi), N unit bins, S ~ U{1..max_slices}."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        n = int(sizes[int(rng.integers(len(sizes)))])
        S = int(rng.integers(1, max_slices + 1))
        jobs.append(dict(n=n, m=3 * n // 2, nd=n, slices=S, seed=1000 * seed + j))
    return jobs


def job_sinograms(job: dict, photons: float = BATCH["photons"],
                  ellipses: int = BATCH["ellipses"]) -> np.ndarray:
    """[S, m, nd] float64 measured sinograms of one batch job: slice s is its
    own random ellipse phantom (seeded by (job seed, s)) with Poisson noise."""
    cs = angle_table(job["m"])
    out = np.empty((job["slices"], job["m"], job["nd"]))
    for s in range(job["slices"]):
        rng = np.random.default_rng([job["seed"], s])
        ells = random_ellipses(rng, ellipses)
        out[s] = poisson_noise(rng, line_integrals(ells, job["n"], cs, job["nd"]), job["n"], photons)
    return out

"""Pins of the oracle's system matrix against geometry and mathematics.

Nothing here compares the oracle with itself: each check uses an independent
construction (closed-form chords, per-pixel clipping, analytic line
integrals of ellipses, hand-derived rows) that a plausible mistake in the
Siddon trace (a dropped crossing, a wrong sign, a transposed pixel index,
a misplaced midpoint) would fail.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2009_07226_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _geom(n, m, nd, offset=0.0, spacing=1.0, cs=None):
    return oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs if cs is not None else inputs.angle_table(m),
                           det_spacing=spacing, det_offset=offset)


# --------------------------------------------------------------------------
# hand-derived rows (tests/golden/siddon_2x2.txt)
# --------------------------------------------------------------------------

def test_golden_2x2_rows():
    with open(os.path.join(GOLDEN, "siddon_2x2.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for fields in rows:
        th = math.radians(float(fields[0]))
        t = float(fields[1])
        want = {int(a.split(":")[0]): float(a.split(":")[1]) for a in fields[2:]}
        col, val = oracle.trace_one(2, math.cos(th), math.sin(th), t)
        got = dict(zip(col.tolist(), val.tolist()))
        assert sorted(got) == sorted(want), (fields, got)
        for c in want:
            assert abs(got[c] - want[c]) <= 1e-12, (fields, got)


# --------------------------------------------------------------------------
# special angles
# --------------------------------------------------------------------------

def test_theta_zero_rows_are_unit_columns():
    """At theta = 0 the rays are vertical lines through pixel-column centres:
    each row holds n entries of exactly 1.0 in column ix = j, and A x is the
    column sums of the image, exactly (integer-valued image)."""
    n = 16
    g = _geom(n, 4, n)
    a = oracle.siddon_csr(g)
    for j in range(n):
        lo, hi = a.rowptr[j], a.rowptr[j + 1]
        assert hi - lo == n
        assert np.all(a.val[lo:hi] == 1.0)
        assert np.all(a.col[lo:hi] % n == j)
        assert sorted((a.col[lo:hi] // n).tolist()) == list(range(n))
    rng = np.random.default_rng(0)
    img = rng.integers(-50, 50, size=(n, n)).astype(np.float64)
    y = oracle.project(a, img.reshape(1, -1))[0]
    assert np.array_equal(y[:n], img.sum(axis=0))


def test_theta_half_pi_is_row_sums():
    n, m = 16, 4                      # theta_2 = pi/2
    g = _geom(n, m, n)
    a = oracle.siddon_csr(g)
    rng = np.random.default_rng(1)
    img = rng.uniform(-1, 1, size=(n, n))
    y = oracle.project(a, img.reshape(1, -1))[0].reshape(m, n)
    # normal (cos, sin) = (~0, 1): ray j is the line y = t_j, i.e. pixel row j
    np.testing.assert_allclose(y[2], img.sum(axis=1), rtol=0, atol=1e-12)


def test_boundary_line_goes_to_higher_pixel():
    """A ray lying exactly on a pixel boundary (theta = 0, integer t) keeps its
    full chord; the midpoint rule puts it in the half-open cell above."""
    n = 8
    col, val = oracle.trace_one(n, 1.0, 0.0, -1.0)
    assert np.all(col % n == 3)          # x = -1 is the left edge of ix = 3
    assert abs(val.sum() - n) < 1e-12


# --------------------------------------------------------------------------
# row sums = chord of the line through the grid square
# --------------------------------------------------------------------------

def _chord_through_square(c, s, t, h):
    """Length of {P . (c, s) = t} inside [-h, h]^2 from the signed distances
    of the square's corners: the line meets the edges whose endpoints lie on
    opposite sides; the chord joins the extreme meeting points."""
    corners = [(-h, -h), (h, -h), (h, h), (-h, h)]
    pts = []
    for i in range(4):
        (x0, y0), (x1, y1) = corners[i], corners[(i + 1) % 4]
        f0 = x0 * c + y0 * s - t
        f1 = x1 * c + y1 * s - t
        if f0 == 0.0:
            pts.append((x0, y0))
        if (f0 < 0 < f1) or (f1 < 0 < f0):
            u = f0 / (f0 - f1)
            pts.append((x0 + u * (x1 - x0), y0 + u * (y1 - y0)))
    best = 0.0
    for i in range(len(pts)):
        for k in range(i + 1, len(pts)):
            best = max(best, math.hypot(pts[i][0] - pts[k][0], pts[i][1] - pts[k][1]))
    return best


@pytest.mark.parametrize("n,m,nd,offset,spacing", [
    (16, 37, 23, 0.0, 1.0), (33, 29, 47, 0.21, 0.77), (64, 64, 64, 0.0, 1.0), (9, 50, 15, -0.3, 1.3)])
def test_row_sums_are_chords(n, m, nd, offset, spacing):
    g = _geom(n, m, nd, offset, spacing)
    a = oracle.siddon_csr(g)
    sums = np.array([a.val[a.rowptr[r]:a.rowptr[r + 1]].sum() for r in range(a.nrow)])
    cs = g.table()
    for r in range(a.nrow):
        k, j = divmod(r, nd)
        t = (j - 0.5 * (nd - 1)) * spacing + offset
        want = _chord_through_square(cs[k, 0], cs[k, 1], t, n / 2)
        tol = 1e-12 * max(want, 1.0) + (2 * n + 2) * 1e-9
        assert abs(sums[r] - want) <= tol, (r, sums[r], want)


# --------------------------------------------------------------------------
# dense brute force: clip the line against every pixel
# --------------------------------------------------------------------------

def _clip_len(px, py, dx, dy, x0, x1, y0, y1):
    """Length of P(a) = p + a d inside [x0,x1] x [y0,y1] (|d| = 1)."""
    lo, hi = -math.inf, math.inf
    for p, d, b0, b1 in ((px, dx, x0, x1), (py, dy, y0, y1)):
        if d == 0.0:
            if not (b0 <= p <= b1):
                return 0.0
            continue
        a0, a1 = (b0 - p) / d, (b1 - p) / d
        lo = max(lo, min(a0, a1))
        hi = min(hi, max(a0, a1))
    return max(0.0, hi - lo)


@pytest.mark.parametrize("offset", [0.0, 0.137, -0.41])
def test_dense_bruteforce_8x8(offset):
    n, m, nd = 8, 8, 8
    cs = inputs.angle_table(m)
    # angles off the axes so no ray lies on a pixel boundary
    th = (np.arange(m) + 0.23) * math.pi / m
    cs = np.stack([np.cos(th), np.sin(th)], axis=1)
    g = _geom(n, m, nd, offset, 1.0, cs)
    a = oracle.siddon_csr(g).to_dense()
    h = n / 2
    ref = np.zeros_like(a)
    for k in range(m):
        c, s = cs[k]
        for j in range(nd):
            t = (j - 0.5 * (nd - 1)) + offset
            for iy in range(n):
                for ix in range(n):
                    ref[k * nd + j, iy * n + ix] = _clip_len(
                        t * c, t * s, -s, c, ix - h, ix - h + 1, iy - h, iy - h + 1)
    big = (ref >= 1e-9) | (a >= 1e-9)
    assert np.array_equal(ref >= 1e-9, a >= 1e-9)
    np.testing.assert_allclose(a[big], ref[big], rtol=0, atol=1e-12)
    assert np.all(a[~big] == 0.0)


# --------------------------------------------------------------------------
# analytic line integrals of ellipse phantoms
# --------------------------------------------------------------------------

def test_ellipse_projections_converge():
    rng = np.random.default_rng(11)
    ells = inputs.random_ellipses(rng, 6, (0.2, 1.0))
    errs = []
    for n in (64, 128, 256):
        g = _geom(n, n, n)
        a = oracle.siddon_csr(g)
        img = inputs.rasterize(ells, n)
        y = oracle.project(a, img.reshape(1, -1))[0]
        want = inputs.line_integrals(ells, n, g.table(), n).reshape(-1)
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    # the rasterised phantom differs from the continuous one along the
    # ellipse edges only, so the error falls as 1/n: a dropped crossing or a
    # misplaced pixel would leave an O(1) error that does not shrink
    assert errs[1] < 3e-2, errs
    for coarse, fine in zip(errs, errs[1:]):
        assert 1.6 < coarse / fine < 2.5, errs


def test_disk_chord_exact_centre_ray():
    """A centred disk of radius R: the central ray's chord is 2R; the
    discrete row through the disk's pixels approaches it as n grows."""
    for n in (64, 256):
        g = _geom(n, 3, n + 1)            # odd bin count: bin n/2 has t = 0
        a = oracle.siddon_csr(g)
        ells = np.array([[0.0, 0.0, 0.5, 0.5, 0.0, 1.0]])
        img = inputs.rasterize(ells, n)
        y = oracle.project(a, img.reshape(1, -1))[0].reshape(3, n + 1)
        assert abs(y[0, n // 2] - n / 2) <= 2.0


# --------------------------------------------------------------------------
# transpose and adjointness
# --------------------------------------------------------------------------

def test_transpose_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    g = _geom(20, 17, 27, 0.3)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    ref = sp.csr_matrix((a.val, a.col, a.rowptr), shape=(a.nrow, a.ncol)).T.tocsr()
    ref.sort_indices()
    assert np.array_equal(at.rowptr, ref.indptr)
    assert np.array_equal(at.col, ref.indices)
    assert np.array_equal(at.val, ref.data)


def test_matrix_free_adjoint():
    """<A x, y> = <x, A^T y> with the projection and back projection each
    computed matrix-free by independent traversals (rays vs pixels)."""
    g = _geom(24, 19, 31, -0.37, 0.9)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, g.npix))
    y = rng.standard_normal((2, g.nrays))
    ax = oracle.project_rays(g, x)
    aty = oracle.backproject_pixels(g, y, np.arange(g.npix))
    lhs = np.einsum("ij,ij->i", ax, y)
    rhs = np.einsum("ij,ij->i", x, aty)
    scale = np.linalg.norm(ax, axis=1) * np.linalg.norm(y, axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)
    a = oracle.siddon_csr(g)
    np.testing.assert_allclose(oracle.project(a, x), ax, rtol=0, atol=1e-12)
    at = oracle.transpose(a)
    np.testing.assert_allclose(oracle.backproject(at, y), aty, rtol=0, atol=1e-11)


@pytest.mark.parametrize("n,m,nd,off,sp", [(8, 8, 8, 0.0, 1.0), (24, 19, 31, -0.37, 0.9),
                                            (37, 23, 41, -0.4, 1.0), (8, 5, 4, 100.0, 1.0)])
def test_ray_scatter_back_projection(n, m, nd, off, sp):
    """The matrix-free back projection by rays (each ray's lengths scattered
    into its pixels) equals the product with the explicit transpose, equals
    the pixel-driven one, and is the adjoint of the ray-driven projection --
    three independent traversals of A."""
    g = _geom(n, m, nd, off, sp)
    rng = np.random.default_rng(n + m)
    x = rng.standard_normal((3, g.npix))
    y = rng.standard_normal((3, g.nrays))
    aty = oracle.backproject_rays(g, y)
    at = oracle.transpose(oracle.siddon_csr(g))
    np.testing.assert_allclose(aty, oracle.backproject(at, y), rtol=0, atol=1e-12 * max(1.0, np.abs(aty).max()))
    np.testing.assert_allclose(aty, oracle.backproject_pixels(g, y, np.arange(g.npix)), rtol=0,
                               atol=1e-11 * max(1.0, np.abs(aty).max()))
    ax = oracle.project_rays(g, x)
    lhs = np.einsum("ij,ij->i", ax, y)
    rhs = np.einsum("ij,ij->i", x, aty)
    scale = np.linalg.norm(ax, axis=1) * np.linalg.norm(y, axis=1) + 1e-300
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


def test_empty_and_degenerate_geometries():
    # all rays miss the grid
    g = _geom(8, 5, 4, offset=100.0)
    a = oracle.siddon_csr(g)
    assert a.nnz == 0 and a.rowptr.shape == (21,)
    # one pixel, one angle, one bin through the centre
    g = _geom(1, 1, 1)
    a = oracle.siddon_csr(g)
    assert a.nnz == 1 and a.col[0] == 0 and a.val[0] == 1.0

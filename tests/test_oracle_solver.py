"""Pins of the oracle's CGLS, Hilbert ordering, rounding model and TV term
against mathematics: Krylov-subspace optimality by dense QR, least-squares
limits, textbook Hilbert curves, IEEE rounding by an independent route, and
finite differences / closed forms for TV."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2009_07226_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_problem(n=8, m=8, nd=8, seed=0, consistent=True):
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=0.11)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    rng = np.random.default_rng(seed)
    xt = rng.uniform(0, 1, size=(2, g.npix))
    b = oracle.project(a, xt)
    if not consistent:
        b = b + 0.05 * rng.standard_normal(b.shape)
    return a, at, b


def _ops(a, at):
    return (lambda X: oracle.project(a, X)), (lambda Y: oracle.backproject(at, Y))


def test_cgls_equals_krylov_minimiser():
    """In exact arithmetic x_k minimises ||b - A x|| over the Krylov space
    K_k(A^T A, A^T b).  The space is built with an orthonormal basis (Gram-
    Schmidt applied twice) and the minimiser found by dense least squares."""
    a, at, b = _small_problem(consistent=False)
    A = a.to_dense()
    A_op, At_op = _ops(a, at)
    # A here is rank-deficient (cond ~ 1e16), so the floating-point Krylov
    # basis drifts by ~10x per step; up to k = 8 both stay within 1e-10
    for k in range(1, 9):
        x, _ = oracle.cgls(A_op, At_op, b, k)
        for s in range(b.shape[0]):
            v = A.T @ b[s]
            basis = []
            for _ in range(k):
                w = v.copy()
                for _rep in range(2):
                    for q in basis:
                        w -= (q @ w) * q
                basis.append(w / np.linalg.norm(w))
                v = A.T @ (A @ basis[-1])
            V = np.stack(basis, axis=1)
            c, *_ = np.linalg.lstsq(A @ V, b[s], rcond=None)
            ref = V @ c
            assert np.linalg.norm(x[s] - ref) <= 1e-9 * np.linalg.norm(ref), (k, s)


def test_cgls_residual_monotone_and_normal_residual_vanishes():
    a, at, b = _small_problem(consistent=True)
    A_op, At_op = _ops(a, at)
    x, log = oracle.cgls(A_op, At_op, b, 200)
    r = log[:, :, 0]
    assert np.all(np.diff(r, axis=0) <= 1e-12 * r[:-1])
    assert np.all(log[-1, :, 1] <= 1e-6 * log[0, :, 1])


def test_cgls_reaches_minimum_norm_least_squares():
    a, at, b = _small_problem(consistent=False, seed=3)
    A = a.to_dense()
    A_op, At_op = _ops(a, at)
    x, log = oracle.cgls(A_op, At_op, b, 400)
    for s in range(b.shape[0]):
        ref = np.linalg.lstsq(A, b[s], rcond=None)[0]
        assert np.linalg.norm(x[s] - ref) <= 1e-6 * np.linalg.norm(ref)
        assert abs(log[-1, s, 0] - np.linalg.norm(b[s] - A @ ref)) <= 1e-8 * np.linalg.norm(b[s])


def test_cgls_counts_one_initial_back_projection():
    """K iterations = K projections and K + 1 back projections (Table IV
    footnote: 30 and 31 for 30 iterations)."""
    a, at, b = _small_problem()
    calls = {"A": 0, "At": 0}

    def A_op(X):
        calls["A"] += 1
        return oracle.project(a, X)

    def At_op(Y):
        calls["At"] += 1
        return oracle.backproject(at, Y)

    oracle.cgls(A_op, At_op, b, 30)
    assert calls == {"A": 30, "At": 31}


def test_cgls_zero_data_stops_cleanly():
    a, at, b = _small_problem()
    A_op, At_op = _ops(a, at)
    b[1] = 0.0
    x, log = oracle.cgls(A_op, At_op, b, 5)
    assert np.all(x[1] == 0.0) and np.all(np.isfinite(x))
    assert np.all(log[:, 1, :] == 0.0)


# --------------------------------------------------------------------------
# Hilbert ordering
# --------------------------------------------------------------------------

def test_hilbert_golden_4x4():
    with open(os.path.join(GOLDEN, "hilbert_4x4.txt")) as f:
        rows = [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    for d, x, y in rows:
        assert oracle.hilbert_index(4, x, y) == d


@pytest.mark.parametrize("side", [2, 4, 8, 32])
def test_hilbert_curve_is_adjacent_walk(side):
    pos = {}
    for y in range(side):
        for x in range(side):
            pos[oracle.hilbert_index(side, x, y)] = (x, y)
    assert sorted(pos) == list(range(side * side))
    for d in range(side * side - 1):
        (x0, y0), (x1, y1) = pos[d], pos[d + 1]
        assert abs(x0 - x1) + abs(y0 - y1) == 1
    assert pos[0] == (0, 0) and pos[side * side - 1] == (side - 1, 0)


@pytest.mark.parametrize("inner", ["row", "col", "quad"])
@pytest.mark.parametrize("nx,ny,tile", [(16, 16, 8), (13, 7, 4), (128, 180, 8), (5, 5, 8), (1, 1, 8),
                                        (10, 6, 4)])
def test_hilbert_order_tiles(nx, ny, tile, inner):
    perm = oracle.hilbert_order(nx, ny, tile, inner)
    assert sorted(perm.tolist()) == list(range(nx * ny))
    grid = perm.reshape(ny, nx)
    # every tile holds a contiguous id range, numbered as `inner` says
    for ty in range(0, ny, tile):
        for tx in range(0, nx, tile):
            blk = grid[ty:ty + tile, tx:tx + tile]
            h, w = blk.shape
            rel = blk - blk.min()
            assert sorted(rel.reshape(-1).tolist()) == list(range(h * w))
            if inner == "row" or (inner == "quad" and (h % 2 or w % 2)):
                assert np.array_equal(rel, np.arange(h * w).reshape(h, w))
            elif inner == "col":
                assert np.array_equal(rel, np.arange(h * w).reshape(w, h).T)
            else:
                # ids 4k..4k+3 fill one 2 x 2 square, row-major inside it;
                # the squares themselves row-major
                for k in range(h * w // 4):
                    ys, xs = np.nonzero((rel >= 4 * k) & (rel < 4 * k + 4))
                    y0, x0 = ys.min(), xs.min()
                    assert y0 % 2 == 0 and x0 % 2 == 0
                    assert np.array_equal(rel[y0:y0 + 2, x0:x0 + 2], 4 * k + np.array([[0, 1], [2, 3]]))
                    assert k == (y0 // 2) * (w // 2) + x0 // 2
    # first tile is the one at the origin
    assert grid[0, 0] == 0


# --------------------------------------------------------------------------
# rounding model
# --------------------------------------------------------------------------

def test_round_f16_matches_numpy_cast():
    rng = np.random.default_rng(2)
    x = np.concatenate([
        rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 5, 20000),
        np.array([65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                  1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -0.0, 0.0])])
    got = oracle.round_f16(x)
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, want, equal_nan=True)


def _bf16_by_bits(x32: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 on the bit pattern: keep the high 16 bits,
    adding half an ulp of the kept part minus one, plus the lowest kept bit
    (ties to even)."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_round_bf16_hand_cases_and_bit_route():
    cases = {1.0 + 2.0 ** -8: 1.0, 1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,
             1.0 + 2.0 ** -7: 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,
             -3.0: -3.0, 0.0: 0.0}
    for x, want in cases.items():
        assert oracle.round_bf16(np.array([x]))[0] == want, x
    rng = np.random.default_rng(3)
    x32 = (rng.standard_normal(50000) * 10.0 ** rng.integers(-30, 30, 50000)).astype(np.float32)
    assert np.array_equal(oracle.round_bf16(x32.astype(np.float64)), _bf16_by_bits(x32))


def test_slice_scale_exponent():
    v = np.array([[0.75, -0.1], [1.0, 0.5], [0.0, 0.0], [-3.0, 2.5], [2.0 ** -30, 0.0]])
    assert oracle.slice_scale_exp(v).tolist() == [0, 0, 0, 2, -30]


def test_mixed_product_exact_on_representable_data():
    """With unit chords (theta = 0) and inputs already representable after
    normalisation, the mixed product equals the exact product."""
    n = 8
    g = oracle.Geometry(n=n, m=1, nd=n, cos_sin=np.array([[1.0, 0.0]]))
    a = oracle.siddon_csr(g)
    rng = np.random.default_rng(4)
    x = rng.integers(-64, 64, size=(3, n * n)).astype(np.float64) / 64.0
    for kind in ("f16", "bf16"):
        np.testing.assert_array_equal(oracle.mixed_project(a, x, kind), oracle.project(a, x))


def test_mixed_product_error_scale():
    """Error of the mixed product relative to FP64 sits at the 16-bit unit
    roundoff (2^-11 for f16, 2^-8 for bf16) and not far below or above."""
    g = oracle.Geometry(n=32, m=24, nd=32, cos_sin=inputs.angle_table(24))
    a = oracle.siddon_csr(g)
    rng = np.random.default_rng(7)
    x = rng.uniform(0.1, 1.0, size=(2, g.npix))
    y = oracle.project(a, x)
    for kind, u in (("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)):
        err = np.linalg.norm(oracle.mixed_project(a, x, kind) - y) / np.linalg.norm(y)
        assert u / 100 < err < u, (kind, err)


def test_matrix16_product_pins():
    """Matrix-only rounding: exact for unit chords and any single-precision
    input; equal to the mixed product when the inputs are already 16-bit
    representable after normalisation; otherwise between the exact product
    and the mixed one, with an error at the matrix's unit roundoff."""
    n = 8
    g0 = oracle.Geometry(n=n, m=1, nd=n, cos_sin=np.array([[1.0, 0.0]]))
    a0 = oracle.siddon_csr(g0)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((3, n * n)).astype(np.float32).astype(np.float64)
    for kind in ("f16", "bf16"):
        np.testing.assert_array_equal(oracle.matrix16_project(a0, x, kind), oracle.project(a0, x))
    g = oracle.Geometry(n=32, m=24, nd=32, cos_sin=inputs.angle_table(24))
    a = oracle.siddon_csr(g)
    xr = rng.integers(1, 64, size=(2, g.npix)).astype(np.float64) / 64.0
    xf = rng.uniform(0.1, 1.0, size=(2, g.npix)).astype(np.float32).astype(np.float64)
    y = oracle.project(a, xf)
    for kind, u in (("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)):
        np.testing.assert_allclose(oracle.matrix16_project(a, xr, kind), oracle.mixed_project(a, xr, kind),
                                   rtol=1e-15, atol=0)
        em = np.linalg.norm(oracle.matrix16_project(a, xf, kind) - y) / np.linalg.norm(y)
        ex = np.linalg.norm(oracle.mixed_project(a, xf, kind) - y) / np.linalg.norm(y)
        assert u / 100 < em < u and em < ex, (kind, em, ex)


# --------------------------------------------------------------------------
# smoothed total variation
# --------------------------------------------------------------------------

def test_tv_closed_forms():
    eps = 1e-3
    n = 6
    val, g = oracle.tv_value_grad(np.full((2, n, n), 3.7), eps)
    assert abs(val - 2 * n * n * eps) < 1e-15
    assert np.all(g == 0.0)
    a = 0.3
    ramp = np.tile(a * np.arange(n, dtype=np.float64), (n, 1))[None]
    val, _ = oracle.tv_value_grad(ramp, eps)
    want = n * (n - 1) * math.sqrt(a * a + eps * eps) + n * eps
    assert abs(val - want) < 1e-12


def test_tv_gradient_by_central_differences():
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, size=(2, 7, 7))
    eps = 1e-3
    _, g = oracle.tv_value_grad(x, eps)
    h = 1e-6
    fd = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd[idx] = (oracle.tv_value_grad(xp, eps)[0] - oracle.tv_value_grad(xm, eps)[0]) / (2 * h)
    assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)

"""Plain CPU FP64 oracle for the memoized parallel-beam XCT projector.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2009_07226_gb300``) and never imports
it; the only module both sides use is the seeded input generator
``paper_2009_07226_gb300.inputs``, which holds none of the method's
arithmetic.

What it computes, each step following the paper:

* ``siddon_csr``      -- the system matrix A: Siddon ray-pixel intersection
  lengths (Sec. II-A), one row per ray, natural order, columns ascending.
  The C trace is in ``xct_oracle.c``.
* ``project`` / ``backproject`` -- Y = A X and X = A^T Y for a batch of slices
  sharing A (Sec. II-B: every ray u_{*,j} traces the same voxels in all
  slices; Sec. III-B2: the fused product A X = B).
* ``project_rays`` / ``backproject_pixels`` -- the same products,
  matrix-free, for a sample of rows (large grids); ``backproject_rays`` --
  the full back projection, matrix-free, as the scatter of every ray.
* ``cgls``            -- least squares on A x = y (Eq. 1 with R = 0 and no
  constraint), in the CGLS form whose K iterations cost K projections and
  K + 1 back projections (Table IV footnote: 30 projections, 31 back
  projections for 30 iterations).
* ``hilbert_order``   -- pseudo-Hilbert ordering of square tiles
  (Sec. III-A1): tiles ordered along the Hilbert curve, row-major inside.
* ``round_f16`` / ``round_bf16`` / ``mixed_project`` -- the mixed-precision
  semantics (Sec. III-C): 16-bit storage of matrix and input vectors with a
  power-of-two normalisation, products summed wide, output de-normalised.
* ``tv_value_grad``   -- a smoothed isotropic total variation R(x) for Eq. 1
  (the paper leaves R unspecified: sum of sqrt(dx^2 + dy^2 + eps^2) with
  forward differences, 0 past the last row / column).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xct_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part with gcc (no FMA contraction, OpenMP over rows)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ci, cd, c64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.orc_siddon_count.argtypes = [ci, ci, ci, f64p, cd, cd, cd, i64p]
        lib.orc_siddon_count.restype = c64
        lib.orc_siddon_fill.argtypes = [ci, ci, ci, f64p, cd, cd, cd, i64p, i32p, f64p]
        lib.orc_siddon_fill.restype = ci
        lib.orc_csr_mm.argtypes = [c64, c64, i64p, i32p, f64p, ci, f64p, f64p]
        lib.orc_csr_mm.restype = None
        lib.orc_csr_transpose.argtypes = [c64, c64, i64p, i32p, f64p, i64p, i32p, f64p]
        lib.orc_csr_transpose.restype = None
        lib.orc_project_rays.argtypes = [ci, ci, ci, f64p, cd, cd, cd, ci, f64p,
                                         ctypes.c_void_p, c64, f64p]
        lib.orc_project_rays.restype = ci
        lib.orc_backproject_pixels.argtypes = [ci, ci, ci, f64p, cd, cd, cd, ci, f64p,
                                               i64p, c64, f64p]
        lib.orc_backproject_pixels.restype = ci
        lib.orc_backproject_rays.argtypes = [ci, ci, ci, f64p, cd, cd, cd, ci, f64p, f64p]
        lib.orc_backproject_rays.restype = ci
        lib.orc_trace_one.argtypes = [ci, cd, cd, cd, cd, i32p, f64p]
        lib.orc_trace_one.restype = ci
        lib.orc_set_threads.argtypes = [ci]
        lib.orc_set_threads.restype = ci
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the C part's OpenMP loops (0: leave as is); returns the
    previous count."""
    return int(_load().orc_set_threads(int(n)))


# --------------------------------------------------------------------------
# Geometry (Sec. II-A gives no conventions: unit pixels centred on the
# origin, ray (k, j) at offset t_j along the normal (cos, sin) of theta_k,
# traversed along (-sin, cos))
# --------------------------------------------------------------------------

def default_angles(m: int) -> np.ndarray:
    """cos/sin of theta_k = k*pi/m, k < m, evaluated with the C library's
    cos and sin (Python's math module) -- [m, 2] float64."""
    cs = np.empty((m, 2), dtype=np.float64)
    for k in range(m):
        th = k * math.pi / m
        cs[k, 0] = math.cos(th)
        cs[k, 1] = math.sin(th)
    return cs


@dataclass
class Geometry:
    n: int                       # grid side, unit pixels, centred at the origin
    m: int                       # angles
    nd: int                      # detector bins
    cos_sin: np.ndarray | None = None
    det_spacing: float = 1.0
    det_offset: float = 0.0
    min_seg: float = 1e-9

    def table(self) -> np.ndarray:
        if self.cos_sin is None:
            self.cos_sin = default_angles(self.m)
        return np.ascontiguousarray(self.cos_sin, dtype=np.float64).reshape(self.m, 2)

    @property
    def nrays(self) -> int:
        return self.m * self.nd

    @property
    def npix(self) -> int:
        return self.n * self.n


@dataclass
class CSR:
    nrow: int
    ncol: int
    rowptr: np.ndarray   # int64 [nrow + 1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrow, self.ncol))
        for r in range(self.nrow):
            lo, hi = self.rowptr[r], self.rowptr[r + 1]
            d[r, self.col[lo:hi]] = self.val[lo:hi]
        return d


def siddon_csr(g: Geometry) -> CSR:
    """A as CSR in natural order (rows = rays k*nd+j, cols = pixels iy*n+ix),
    columns ascending inside each row (Siddon, Sec. II-A)."""
    lib = _load()
    cs = g.table()
    cnt = np.zeros(g.nrays, dtype=np.int64)
    dup = lib.orc_siddon_count(g.n, g.m, g.nd, cs.reshape(-1), g.det_spacing,
                               g.det_offset, g.min_seg, cnt)
    if dup != 0:
        raise RuntimeError(f"Siddon trace produced {dup} duplicate pixels (or failed)")
    rowptr = np.zeros(g.nrays + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(max(nnz, 1), dtype=np.int32)
    val = np.empty(max(nnz, 1), dtype=np.float64)
    if lib.orc_siddon_fill(g.n, g.m, g.nd, cs.reshape(-1), g.det_spacing,
                           g.det_offset, g.min_seg, rowptr, col, val) != 0:
        raise RuntimeError("Siddon fill failed")
    return CSR(g.nrays, g.npix, rowptr, col[:nnz].copy(), val[:nnz].copy())


def trace_one(n: int, c: float, s: float, t: float, min_seg: float = 1e-9):
    """Entries (cols, lengths) of one ray with normal (c, s) at offset t."""
    lib = _load()
    col = np.empty(2 * n + 4, dtype=np.int32)
    val = np.empty(2 * n + 4, dtype=np.float64)
    k = lib.orc_trace_one(n, c, s, t, min_seg, col, val)
    if k < 0:
        raise MemoryError
    return col[:k].copy(), val[:k].copy()


def transpose(a: CSR) -> CSR:
    """A^T as CSR (stable: entries of each column keep ascending ray order)."""
    lib = _load()
    nnz = a.nnz
    trp = np.empty(a.ncol + 1, dtype=np.int64)
    tcol = np.empty(max(nnz, 1), dtype=np.int32)
    tval = np.empty(max(nnz, 1), dtype=np.float64)
    col = a.col if nnz else np.zeros(1, np.int32)
    val = a.val if nnz else np.zeros(1, np.float64)
    lib.orc_csr_transpose(a.nrow, a.ncol, a.rowptr, col, val, trp, tcol, tval)
    return CSR(a.ncol, a.nrow, trp, tcol[:nnz].copy(), tval[:nnz].copy())


def csr_mm(a: CSR, X: np.ndarray) -> np.ndarray:
    """Y = A X with slice-major X [S, ncol] -> Y [S, nrow], FP64."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, a.ncol)
    S = X.shape[0]
    Y = np.empty((S, a.nrow), dtype=np.float64)
    col = a.col if a.nnz else np.zeros(1, np.int32)
    val = a.val if a.nnz else np.zeros(1, np.float64)
    if X.size == 0:
        return Y
    lib.orc_csr_mm(a.nrow, a.ncol, a.rowptr, col, val, S, X, Y)
    return Y


def project(a: CSR, X: np.ndarray) -> np.ndarray:
    """Projection Y = A X (Sec. II-A forward operator), slice-major."""
    return csr_mm(a, X)


def backproject(at: CSR, Y: np.ndarray) -> np.ndarray:
    """Back projection X = A^T Y using the explicit transpose."""
    return csr_mm(at, Y)


def project_rays(g: Geometry, X: np.ndarray, rays=None) -> np.ndarray:
    """Matrix-free projection of the listed natural ray ids (all if None)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, g.npix)
    S = X.shape[0]
    if rays is None:
        count, ptr = g.nrays, None
    else:
        rays = np.ascontiguousarray(rays, dtype=np.int64)
        count, ptr = rays.size, rays.ctypes.data
    Y = np.empty((S, count), dtype=np.float64)
    if count and S:
        if lib.orc_project_rays(g.n, g.m, g.nd, g.table().reshape(-1), g.det_spacing,
                                g.det_offset, g.min_seg, S, X, ptr, count, Y):
            raise MemoryError
    return Y


def backproject_pixels(g: Geometry, Y: np.ndarray, pixels) -> np.ndarray:
    """Matrix-free back projection for the listed natural pixel ids."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, g.nrays)
    S = Y.shape[0]
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    X = np.empty((S, pixels.size), dtype=np.float64)
    if pixels.size and S:
        if lib.orc_backproject_pixels(g.n, g.m, g.nd, g.table().reshape(-1),
                                      g.det_spacing, g.det_offset, g.min_seg, S, Y,
                                      pixels, pixels.size, X):
            raise MemoryError
    return X


def backproject_rays(g: Geometry, Y: np.ndarray) -> np.ndarray:
    """Matrix-free back projection X = A^T Y over all rays: every ray traced
    again and its segment lengths scattered, x[pixel] += length * y[ray]
    (the transpose product by its definition, for grids whose A does not
    fit in host memory)."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, g.nrays)
    S = Y.shape[0]
    X = np.empty((S, g.npix), dtype=np.float64)
    if S and g.nrays:
        if lib.orc_backproject_rays(g.n, g.m, g.nd, g.table().reshape(-1), g.det_spacing,
                                    g.det_offset, g.min_seg, S, Y, X):
            raise MemoryError
    elif S:
        X[:] = 0.0
    return X


# --------------------------------------------------------------------------
# CGLS (Eq. 1 with R = 0, unconstrained; per-slice scalars)
# --------------------------------------------------------------------------

def cgls(A, At, b: np.ndarray, iters: int, x0: np.ndarray | None = None):
    """CGLS on each slice independently.

    A(X) and At(Y) apply the operator to slice-major batches.  b is [S, R].
    Returns (x [S, C], log [iters + 1, S, 2]) where log[k, s] holds
    (||r_k||, ||A^T r_k||) after iteration k (k = 0: the start).

    Recurrence (one initial back projection, then one projection and one
    back projection per iteration):
        r = b - A x;  s = A^T r;  p = s;  gamma = ||s||^2
        repeat: q = A p;  delta = ||q||^2;  alpha = gamma / delta
                x += alpha p;  r -= alpha q;  s = A^T r
                gamma' = ||s||^2;  beta = gamma' / gamma;  p = s + beta p
    A slice whose gamma or delta is exactly 0 stops (alpha = 0 from then on).
    """
    b = np.asarray(b, dtype=np.float64)
    S = b.shape[0]
    if x0 is None:
        r = b.copy()
        x = None
    else:
        x = np.array(x0, dtype=np.float64, copy=True)
        r = b - A(x)
    s = At(r)
    if x is None:
        x = np.zeros_like(s)
    p = s.copy()
    gamma = np.einsum("ij,ij->i", s, s)
    active = gamma > 0
    log = np.zeros((iters + 1, S, 2))
    log[0, :, 0] = np.sqrt(np.einsum("ij,ij->i", r, r))
    log[0, :, 1] = np.sqrt(gamma)
    for k in range(1, iters + 1):
        q = A(p)
        delta = np.einsum("ij,ij->i", q, q)
        active &= delta > 0
        alpha = np.where(active, gamma / np.where(delta > 0, delta, 1.0), 0.0)
        x += alpha[:, None] * p
        r -= alpha[:, None] * q
        s = At(r)
        gnew = np.einsum("ij,ij->i", s, s)
        beta = np.where(active, gnew / np.where(gamma > 0, gamma, 1.0), 0.0)
        p = s + beta[:, None] * p
        gamma = np.where(active, gnew, gamma)
        active &= gnew > 0
        log[k, :, 0] = np.sqrt(np.einsum("ij,ij->i", r, r))
        log[k, :, 1] = np.sqrt(gnew)
    return x, log


# --------------------------------------------------------------------------
# Pseudo-Hilbert tile ordering (Sec. III-A1)
# --------------------------------------------------------------------------

def hilbert_index(side: int, x: int, y: int) -> int:
    """Position of cell (x, y) along the Hilbert curve filling a side x side
    grid (side a power of two).  Order-1 curve: (0,0),(0,1),(1,1),(1,0).

    At each level the quadrant (rx, ry) fixes two bits of the position
    (quadrant rank (3*rx) ^ ry), then the coordinates are reduced into the
    quadrant and reflected/transposed so that the sub-curve starts where the
    parent curve enters the quadrant."""
    d = 0
    s = side // 2
    while s > 0:
        rx = 1 if (x & s) else 0
        ry = 1 if (y & s) else 0
        d += s * s * ((3 * rx) ^ ry)
        x &= s - 1
        y &= s - 1
        if ry == 0:
            if rx == 1:
                x = s - 1 - x
                y = s - 1 - y
            x, y = y, x
        s //= 2
    return d


def hilbert_order(nx: int, ny: int, tile: int, inner: str = "row") -> np.ndarray:
    """Map natural id (y * nx + x) -> ordered id.  Cells are grouped in
    tile x tile squares (ragged at the far edges); squares are ordered by
    their Hilbert position on the smallest power-of-two square grid that
    holds them; cells inside a square are numbered by `inner`:
      'row'  -- row-major (x fastest);
      'col'  -- column-major (y fastest);
      'quad' -- 2 x 2 groups of cells, the groups row-major and the cells of
                a group row-major (squares with an odd width or height are
                numbered row-major)."""
    if inner not in ("row", "col", "quad"):
        raise ValueError(inner)
    ntx = -(-nx // tile)
    nty = -(-ny // tile)
    side = 1
    while side < max(ntx, nty):
        side *= 2
    tiles = []
    for ty in range(nty):
        for tx in range(ntx):
            tiles.append((hilbert_index(side, tx, ty), tx, ty))
    tiles.sort()
    perm = np.empty((ny, nx), dtype=np.int64)
    nxt = 0
    for _, tx, ty in tiles:
        x0, y0 = tx * tile, ty * tile
        w = min(tile, nx - x0)
        h = min(tile, ny - y0)
        ly, lx = np.mgrid[0:h, 0:w]
        if inner == "col":
            local = lx * h + ly
        elif inner == "quad" and w % 2 == 0 and h % 2 == 0:
            local = ((ly // 2) * (w // 2) + lx // 2) * 4 + (ly % 2) * 2 + lx % 2
        else:
            local = ly * w + lx
        perm[y0:y0 + h, x0:x0 + w] = nxt + local
        nxt += h * w
    return perm.reshape(-1)


# --------------------------------------------------------------------------
# Mixed precision (Sec. III-C)
# --------------------------------------------------------------------------

def _round_sig(x: np.ndarray, sig_bits: int, min_exp: int, max_finite: float) -> np.ndarray:
    """Round to the nearest value with `sig_bits` significant bits, ties to
    even, with gradual underflow below 2**min_exp (the smallest normal) and
    overflow to infinity above max_finite (IEEE 754 round-to-nearest)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    m, e = np.frexp(np.abs(x[nz]))           # |x| = m * 2**e, m in [0.5, 1)
    # the quantum of a value in [2**(e-1), 2**e) is 2**(e - sig_bits),
    # never finer than the subnormal quantum 2**(min_exp - sig_bits + 1)
    q = np.maximum(e - sig_bits, min_exp - sig_bits + 1)
    mag = np.rint(np.ldexp(np.abs(x[nz]), -q))   # rint: ties to even
    r = np.ldexp(mag, q)
    r = np.where(r > max_finite, np.inf, r)
    out[nz] = np.copysign(r, x[nz])
    return out


def round_f16(x) -> np.ndarray:
    """IEEE binary16 round-to-nearest-even (11 significant bits)."""
    return _round_sig(x, 11, -14, 65504.0)


def round_bf16(x) -> np.ndarray:
    """bfloat16 round-to-nearest-even (8 significant bits, binary32 range)."""
    return _round_sig(x, 8, -126, float(np.float32(3.3895313892515355e38)))


MATRIX_SCALE_EXP = {"f16": 15, "bf16": 0}
_ROUND = {"f16": round_f16, "bf16": round_bf16}


def slice_scale_exp(v: np.ndarray) -> np.ndarray:
    """Per-slice normalisation exponent e = ceil(log2(max |v_s|)) (0 for an
    all-zero slice): v_s * 2**-e then lies in [-1, 1]  (Sec. III-C1,
    adaptive normalisation by the max-norm of the input vector)."""
    v = np.asarray(v).reshape(v.shape[0], -1)
    mx = np.max(np.abs(v), axis=1) if v.shape[1] else np.zeros(v.shape[0])
    out = np.zeros(v.shape[0], dtype=np.int64)
    for s, a in enumerate(mx):
        if a > 0:
            fm, fe = math.frexp(float(a))   # a = fm * 2**fe, fm in [0.5, 1)
            out[s] = fe - 1 if fm == 0.5 else fe
    return out


def mixed_project(a: CSR, X: np.ndarray, kind: str) -> np.ndarray:
    """The mixed-precision product as the paper defines it (Sec. III-C):
    matrix entries stored as RN16(l * 2**k), input slices stored as
    RN16(x * 2**-e_s) from their single-precision values, products of the
    16-bit values summed (here exactly, in FP64), and the sum multiplied by
    2**(e_s - k).  k = 15 for binary16 (largest power of two keeping the
    longest chord sqrt(2) * 2**k below 65504) and 0 for bfloat16."""
    rnd = _ROUND[kind]
    k = MATRIX_SCALE_EXP[kind]
    X32 = np.asarray(X, dtype=np.float32).reshape(-1, a.ncol)
    e = slice_scale_exp(X32)
    Xq = np.empty(X32.shape, dtype=np.float64)
    for s in range(X32.shape[0]):
        scaled = (X32[s] * np.float32(2.0 ** (-int(e[s])))).astype(np.float32)
        Xq[s] = rnd(scaled.astype(np.float64))
    aq = CSR(a.nrow, a.ncol, a.rowptr, a.col, rnd(a.val * 2.0 ** k))
    Y = csr_mm(aq, Xq)
    return Y * (2.0 ** (e.astype(np.float64) - k))[:, None]


def matrix16_project(a: CSR, X: np.ndarray, kind: str) -> np.ndarray:
    """The product with only the matrix in 16 bits (the storage half of Sec.
    III-C): entries RN16(l * 2**k), input slices kept in single precision,
    products summed (here exactly, in FP64) and multiplied by 2**-k.  kind
    'f16' or 'bf16' names the value format."""
    rnd = _ROUND[kind]
    k = MATRIX_SCALE_EXP[kind]
    X32 = np.asarray(X, dtype=np.float32).reshape(-1, a.ncol).astype(np.float64)
    aq = CSR(a.nrow, a.ncol, a.rowptr, a.col, rnd(a.val * 2.0 ** k))
    return csr_mm(aq, X32) * 2.0 ** -k


# --------------------------------------------------------------------------
# Smoothed total variation (a reading of R(x) in Eq. 1)
# --------------------------------------------------------------------------

def tv_value_grad(x: np.ndarray, eps: float):
    """TV_eps(x) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2) per slice with forward
    differences dx = x[i, j+1] - x[i, j], dy = x[i+1, j] - x[i, j] and a
    difference past the last column/row taken as 0 (Neumann boundary).
    x is [S, n, n]; returns (value summed over slices, gradient [S, n, n])."""
    x = np.asarray(x, dtype=np.float64)
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    dy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    mag = np.sqrt(dx * dx + dy * dy + eps * eps)
    val = float(mag.sum())
    ux = dx / mag
    uy = dy / mag
    g = -(ux + uy)
    g[:, :, 1:] += ux[:, :, :-1]
    g[:, 1:, :] += uy[:, :-1, :]
    return val, g


def adam_tv_reconstruct(a: CSR, at: CSR, y: np.ndarray, n: int, steps: int, lr: float, lam: float,
                        eps: float, beta1: float = 0.9, beta2: float = 0.999, adam_eps: float = 1e-8,
                        x0: np.ndarray | None = None):
    """Regularised reconstruction of Eq. 1 with R(x) = lam * TV_eps(x), by the
    gradient iteration of Sec. II-A (project, residual, back project, update)
    with Adam (Kingma & Ba, bias-corrected, no weight decay) as the update.
    Cost summed over slices: sum_s 0.5 ||A x_s - y_s||^2 + lam TV_eps(x_s).
    y is [S, M*N_d]; returns (x [S, n*n], cost before each step [steps]), FP64."""
    y = np.asarray(y, dtype=np.float64)
    S = y.shape[0]
    x = np.zeros((S, n * n)) if x0 is None else np.array(x0, dtype=np.float64).reshape(S, n * n)
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    hist = np.empty(steps)
    for t in range(1, steps + 1):
        r = project(a, x) - y
        tv, tg = tv_value_grad(x.reshape(S, n, n), eps)
        hist[t - 1] = 0.5 * float((r * r).sum()) + lam * tv
        g = backproject(at, r) + lam * tg.reshape(S, -1)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        x = x - lr * mhat / (np.sqrt(vhat) + adam_eps)
    return x, hist

/*
 * Plain CPU FP64 oracle for the memoized parallel-beam projector.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or table with the CUDA
 * library: every number here is computed from the definitions below.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product and sum rounds exactly as written).
 *
 * Geometry (paper Sec. II-A: parallel beam, slices independent; the exact
 * conventions are not given by the paper and are fixed here):
 *   - pixel (ix, iy) of an n x n grid covers [ix - n/2, ix - n/2 + 1] x
 *     [iy - n/2, iy - n/2 + 1]; natural pixel id = iy * n + ix.
 *   - ray (k, j), k < m angles, j < nd bins; natural ray id = k * nd + j.
 *     normal (c, s) = (cos th_k, sin th_k) taken from a caller table,
 *     offset t = (j - (nd - 1) / 2) * dspace + doff, direction (-s, c),
 *     points P(a) = t * (c, s) + a * (-s, c).
 * System matrix (paper Sec. II-A, Siddon's parametric method): the entry
 * A[ray, pixel] is the length of the ray inside the pixel.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Siddon ray trace (classic form).                                          */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x < y) ? -1 : (x > y) ? 1 : 0;
}

typedef struct { int32_t col; double val; } entry_t;

static int cmp_entry(const void* a, const void* b) {
  int32_t x = ((const entry_t*)a)->col, y = ((const entry_t*)b)->col;
  return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/*
 * Trace one ray.  Writes up to 2n+2 entries into `out` (columns ascending)
 * and returns the count; `alpha` is caller scratch of 2n+2 doubles.
 *
 * Steps, in the order of Siddon's method:
 *  1. clip the line against the slabs |x| <= n/2 and |y| <= n/2:
 *     a_min = max of the entry parameters, a_max = min of the exit parameters;
 *     an axis whose direction component is exactly 0.0 gives no parameters,
 *     and the ray misses unless |p_axis| <= n/2 (the grid square is closed:
 *     a line on its edge keeps its chord, assigned by the midpoint rule and
 *     the clamp in step 5);
 *  2. the row is empty unless a_max - a_min >= min_seg;
 *  3. every interior plane (i - n/2, i = 1..n-1) of each axis with a nonzero
 *     direction component is crossed at a = (plane - p) / d, computed directly
 *     from the plane index; crossings strictly inside (a_min, a_max) are kept;
 *  4. {a_min, crossings, a_max} sorted ascending;
 *  5. each consecutive pair gives a segment of length a[m+1] - a[m];
 *     segments shorter than min_seg are dropped; the pixel is the one holding
 *     the segment midpoint, ix = floor(x_mid + n/2) clamped to [0, n-1].
 */
static int trace_ray(int n, double c, double s, double t, double min_seg,
                     double* alpha, entry_t* out) {
  const double half = 0.5 * (double)n;
  const double px = t * c, py = t * s;
  const double dx = -s, dy = c;
  double amin = -INFINITY, amax = INFINITY;

  if (dx != 0.0) {
    double a0 = (-half - px) / dx, a1 = (half - px) / dx;
    double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
    if (lo > amin) amin = lo;
    if (hi < amax) amax = hi;
  } else if (!(fabs(px) <= half)) {
    return 0;
  }
  if (dy != 0.0) {
    double a0 = (-half - py) / dy, a1 = (half - py) / dy;
    double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
    if (lo > amin) amin = lo;
    if (hi < amax) amax = hi;
  } else if (!(fabs(py) <= half)) {
    return 0;
  }
  if (!(amax - amin >= min_seg)) return 0;

  int na = 0;
  alpha[na++] = amin;
  for (int i = 1; i < n; ++i) {
    double plane = (double)i - half;
    if (dx != 0.0) {
      double a = (plane - px) / dx;
      if (a > amin && a < amax) alpha[na++] = a;
    }
    if (dy != 0.0) {
      double a = (plane - py) / dy;
      if (a > amin && a < amax) alpha[na++] = a;
    }
  }
  alpha[na++] = amax;
  qsort(alpha, (size_t)na, sizeof(double), cmp_double);

  int cnt = 0;
  for (int m = 0; m + 1 < na; ++m) {
    double len = alpha[m + 1] - alpha[m];
    if (len < min_seg) continue;
    double mid = (alpha[m] + alpha[m + 1]) * 0.5;
    double x = px + mid * dx;
    double y = py + mid * dy;
    int ix = (int)floor(x + half);
    int iy = (int)floor(y + half);
    if (ix < 0) ix = 0;
    if (ix > n - 1) ix = n - 1;
    if (iy < 0) iy = 0;
    if (iy > n - 1) iy = n - 1;
    out[cnt].col = iy * n + ix;
    out[cnt].val = len;
    ++cnt;
  }
  qsort(out, (size_t)cnt, sizeof(entry_t), cmp_entry);
  return cnt;
}

static double ray_offset(int j, int nd, double dspace, double doff) {
  return ((double)j - 0.5 * (double)(nd - 1)) * dspace + doff;
}

/* Returns -1 on allocation failure, else the number of duplicate columns
 * found inside rows (0 for a valid matrix). */
int64_t orc_siddon_count(int n, int m, int nd, const double* cs, double dspace,
                         double doff, double min_seg, int64_t* rowcount) {
  int64_t dup = 0;
  int fail = 0;
#pragma omp parallel reduction(+ : dup) reduction(| : fail)
  {
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
    entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    if (!alpha || !ent) {
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t r = 0; r < (int64_t)m * nd; ++r) {
        int k = (int)(r / nd), j = (int)(r % nd);
        int c = trace_ray(n, cs[2 * k], cs[2 * k + 1],
                          ray_offset(j, nd, dspace, doff), min_seg, alpha, ent);
        for (int q = 1; q < c; ++q) dup += (ent[q].col == ent[q - 1].col);
        rowcount[r] = c;
      }
    }
    free(alpha);
    free(ent);
  }
  return fail ? -1 : dup;
}

int orc_siddon_fill(int n, int m, int nd, const double* cs, double dspace,
                    double doff, double min_seg, const int64_t* rowptr,
                    int32_t* col, double* val) {
  int fail = 0;
#pragma omp parallel reduction(| : fail)
  {
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
    entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    if (!alpha || !ent) {
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t r = 0; r < (int64_t)m * nd; ++r) {
        int k = (int)(r / nd), j = (int)(r % nd);
        int c = trace_ray(n, cs[2 * k], cs[2 * k + 1],
                          ray_offset(j, nd, dspace, doff), min_seg, alpha, ent);
        if (c != (int)(rowptr[r + 1] - rowptr[r])) { fail = 1; continue; }
        for (int q = 0; q < c; ++q) {
          col[rowptr[r] + q] = ent[q].col;
          val[rowptr[r] + q] = ent[q].val;
        }
      }
    }
    free(alpha);
    free(ent);
  }
  return fail;
}

/* ------------------------------------------------------------------------ */
/* Products with a stored matrix (paper Sec. II-B: one A shared by all        */
/* slices; Sec. III-B2: A X = B with one column of X per slice).             */
/* Vectors are slice-major: X[s * ncol + c], Y[s * nrow + r].                */
/* ------------------------------------------------------------------------ */

/* Y = A X for a CSR matrix; each row sums its entries in stored order. */
void orc_csr_mm(int64_t nrow, int64_t ncol, const int64_t* rowptr,
                const int32_t* col, const double* val, int nslice,
                const double* X, double* Y) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < nrow; ++r) {
    for (int s = 0; s < nslice; ++s) {
      const double* xs = X + (int64_t)s * ncol;
      double acc = 0.0;
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) acc += val[e] * xs[col[e]];
      Y[(int64_t)s * nrow + r] = acc;
    }
  }
}

/* Transpose by a stable counting sort on the column: entries of each output
 * row keep ascending input-row order. */
void orc_csr_transpose(int64_t nrow, int64_t ncol, const int64_t* rowptr,
                       const int32_t* col, const double* val, int64_t* trowptr,
                       int32_t* tcol, double* tval) {
  for (int64_t c = 0; c <= ncol; ++c) trowptr[c] = 0;
  for (int64_t e = 0; e < rowptr[nrow]; ++e) trowptr[col[e] + 1] += 1;
  for (int64_t c = 0; c < ncol; ++c) trowptr[c + 1] += trowptr[c];
  int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncol > 0 ? ncol : 1));
  for (int64_t c = 0; c < ncol; ++c) cursor[c] = trowptr[c];
  for (int64_t r = 0; r < nrow; ++r) {
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      int64_t p = cursor[col[e]]++;
      tcol[p] = (int32_t)r;
      tval[p] = val[e];
    }
  }
  free(cursor);
}

/* ------------------------------------------------------------------------ */
/* Matrix-free forms (the same trace, nothing stored) for grids whose stored */
/* FP64 matrix would not fit in host memory.                                 */
/* ------------------------------------------------------------------------ */

/* Y[s][ray] = sum over the ray's entries of val * X[s][col], for the listed
 * natural ray ids only (all rays when rays == NULL, count = m * nd).  Y is
 * [nslice][count]. */
int orc_project_rays(int n, int m, int nd, const double* cs, double dspace,
                     double doff, double min_seg, int nslice, const double* X,
                     const int64_t* rays, int64_t count, double* Y) {
  int fail = 0;
  (void)m;   /* the ray ids carry the angle; m is kept for a uniform signature */
  const int64_t npix = (int64_t)n * n;
#pragma omp parallel reduction(| : fail)
  {
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
    entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    if (!alpha || !ent) {
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t q = 0; q < count; ++q) {
        int64_t r = rays ? rays[q] : q;
        int k = (int)(r / nd), j = (int)(r % nd);
        int c = trace_ray(n, cs[2 * k], cs[2 * k + 1],
                          ray_offset(j, nd, dspace, doff), min_seg, alpha, ent);
        for (int s = 0; s < nslice; ++s) {
          double acc = 0.0;
          for (int e = 0; e < c; ++e) acc += ent[e].val * X[(int64_t)s * npix + ent[e].col];
          Y[(int64_t)s * count + q] = acc;
        }
      }
    }
    free(alpha);
    free(ent);
  }
  return fail;
}

/* X[s][pixel] = sum over rays crossing the pixel of val * Y[s][ray], for the
 * listed natural pixel ids.  For each angle only the bins whose ray can reach
 * the pixel are traced: the pixel centre projects to t_c = xc*c + yc*s and a
 * ray at offset t can touch the pixel only if |t - t_c| <= (|c| + |s|) / 2;
 * bins within that window plus one on each side are traced in full and the
 * entry for the pixel, if any, is taken.  Sums run over ascending ray id.
 * X is [nslice][count]. */
int orc_backproject_pixels(int n, int m, int nd, const double* cs,
                           double dspace, double doff, double min_seg,
                           int nslice, const double* Y, const int64_t* pixels,
                           int64_t count, double* X) {
  int fail = 0;
  const int64_t nray = (int64_t)m * nd;
#pragma omp parallel reduction(| : fail)
  {
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
    entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(nslice > 0 ? nslice : 1));
    if (!alpha || !ent || !acc) {
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 16)
      for (int64_t q = 0; q < count; ++q) {
        int64_t pix = pixels[q];
        int ix = (int)(pix % n), iy = (int)(pix / n);
        double xc = (double)ix - 0.5 * (double)n + 0.5;
        double yc = (double)iy - 0.5 * (double)n + 0.5;
        for (int s = 0; s < nslice; ++s) acc[s] = 0.0;
        for (int k = 0; k < m; ++k) {
          double c = cs[2 * k], sn = cs[2 * k + 1];
          double tc = xc * c + yc * sn;
          double w = 0.5 * (fabs(c) + fabs(sn));
          /* bin j has t_j = (j - (nd-1)/2) * dspace + doff */
          double jlo = (tc - w - doff) / dspace + 0.5 * (double)(nd - 1);
          double jhi = (tc + w - doff) / dspace + 0.5 * (double)(nd - 1);
          if (dspace < 0) { double tmp = jlo; jlo = jhi; jhi = tmp; }
          int j0 = (int)floor(jlo) - 1, j1 = (int)ceil(jhi) + 1;
          if (j0 < 0) j0 = 0;
          if (j1 > nd - 1) j1 = nd - 1;
          for (int j = j0; j <= j1; ++j) {
            int cnt = trace_ray(n, c, sn, ray_offset(j, nd, dspace, doff),
                                min_seg, alpha, ent);
            for (int e = 0; e < cnt; ++e) {
              if (ent[e].col == (int32_t)pix) {
                int64_t r = (int64_t)k * nd + j;
                for (int s = 0; s < nslice; ++s)
                  acc[s] += ent[e].val * Y[(int64_t)s * nray + r];
                break;
              }
            }
          }
        }
        for (int s = 0; s < nslice; ++s) X[(int64_t)s * count + q] = acc[s];
      }
    }
    free(alpha);
    free(ent);
    free(acc);
  }
  return fail;
}

/* One traced row, for tests: returns the count, fills col/val (ascending). */
/* x = A^T y over all rays, matrix-free (the transpose product written as
 * the scatter of each ray's segments: x[pixel] += length * y[ray]).  Each
 * thread traces a fixed contiguous range of rays into its own buffer; the
 * buffers are summed in thread order.  Returns nonzero on allocation
 * failure. */
int orc_backproject_rays(int n, int m, int nd, const double* cs, double dspace,
                         double doff, double min_seg, int nslice, const double* Y,
                         double* X) {
  const int64_t npix = (int64_t)n * n, nray = (int64_t)m * nd;
  const int nt = omp_get_max_threads();
  double* part = (double*)calloc((size_t)nt * nslice * npix, sizeof(double));
  if (!part) return 1;
  int fail = 0;
#pragma omp parallel num_threads(nt) reduction(| : fail)
  {
    const int t = omp_get_thread_num(), tn = omp_get_num_threads();
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
    entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    double* xt = part + (int64_t)t * nslice * npix;
    if (!alpha || !ent) {
      fail = 1;
    } else {
      const int64_t r0 = nray * t / tn, r1 = nray * (t + 1) / tn;
      for (int64_t r = r0; r < r1; ++r) {
        int k = (int)(r / nd), j = (int)(r % nd);
        int c = trace_ray(n, cs[2 * k], cs[2 * k + 1],
                          ray_offset(j, nd, dspace, doff), min_seg, alpha, ent);
        for (int s = 0; s < nslice; ++s) {
          const double yv = Y[(int64_t)s * nray + r];
          for (int e = 0; e < c; ++e) xt[(int64_t)s * npix + ent[e].col] += ent[e].val * yv;
        }
      }
    }
    free(alpha);
    free(ent);
  }
  if (!fail) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)nslice * npix; ++i) {
      double acc = 0.0;
      for (int t = 0; t < nt; ++t) acc += part[(int64_t)t * nslice * npix + i];
      X[i] = acc;
    }
  }
  free(part);
  return fail;
}

int orc_trace_one(int n, double c, double s, double t, double min_seg,
                  int32_t* col, double* val) {
  double* alpha = (double*)malloc(sizeof(double) * (size_t)(2 * n + 4));
  entry_t* ent = (entry_t*)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
  int cnt = -1;
  if (alpha && ent) {
    cnt = trace_ray(n, c, s, t, min_seg, alpha, ent);
    for (int e = 0; e < cnt; ++e) { col[e] = ent[e].col; val[e] = ent[e].val; }
  }
  free(alpha);
  free(ent);
  return cnt;
}

/* Threads of the OpenMP loops (timing on one core or on all of them);
 * returns the previous setting. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}


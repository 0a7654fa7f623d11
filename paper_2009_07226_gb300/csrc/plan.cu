// Plan construction: the memoized system matrix (paper Sec. II-B).
//
//  1. pseudo-Hilbert orderings of pixels and rays (Sec. III-A1);
//  2. Siddon trace of every ray, count pass + scan + fill pass, FP64 with
//     every product and sum rounded separately (no FMA contraction), so the
//     matrix is bit-identical to a plain sequential evaluation (Sec. II-A);
//  3. the explicit transpose, entries of each column in ascending ray order
//     (Sec. III-B: A and A^T both read from memory);
//  4. the staged kernel layout of each (Sec. III-B1 input buffering,
//     III-B4 multi-stage buffering, III-C2 packed {index, value} entries).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "xct_internal.cuh"

namespace xct {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 0x7fffffffLL) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// 1. pseudo-Hilbert ordering
// ---------------------------------------------------------------------------

// Position of cell (x, y) on the Hilbert curve of a side x side grid (side a
// power of two), orientation (0,0),(0,1),(1,1),(1,0) at order 1: at every
// level the quadrant contributes s*s*((3*rx)^ry); the curve inside a lower
// quadrant is the parent transposed (left) or anti-transposed (right).
__device__ int64_t hilbert_pos(int64_t side, int64_t x, int64_t y) {
  int64_t d = 0;
  for (int64_t s = side >> 1; s > 0; s >>= 1) {
    int rx = (x & s) ? 1 : 0;
    int ry = (y & s) ? 1 : 0;
    d += s * s * (int64_t)((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = side - 1 - x;
        y = side - 1 - y;
      }
      int64_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

// numbering inside a tile
constexpr int kInnerRow = 0;    // x fastest
constexpr int kInnerCol = 1;    // y fastest
constexpr int kInnerQuad = 2;   // 2 x 2 groups, row-major (row-major if a side is odd)

__global__ void tile_sizes_kernel(int64_t nx, int64_t ny, int64_t T, int64_t ntx, int64_t nty,
                                  int64_t side, int64_t* tile_size) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ntx * nty) return;
  int64_t tx = i % ntx, ty = i / ntx;
  int64_t w = min(T, nx - tx * T), h = min(T, ny - ty * T);
  tile_size[hilbert_pos(side, tx, ty)] = w * h;
}

__global__ void order_kernel(int64_t nx, int64_t ny, int64_t T, int64_t side, int inner,
                             const int64_t* tile_off, int32_t* order, int32_t* inv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nx * ny) return;
  int64_t x = i % nx, y = i / nx;
  int64_t tx = x / T, ty = y / T;
  int64_t w = min(T, nx - tx * T), h = min(T, ny - ty * T);
  int64_t lx = x - tx * T, ly = y - ty * T;
  int64_t local;
  if (inner == kInnerCol)
    local = lx * h + ly;
  else if (inner == kInnerQuad && w % 2 == 0 && h % 2 == 0)
    local = ((ly / 2) * (w / 2) + lx / 2) * 4 + (ly % 2) * 2 + lx % 2;
  else
    local = ly * w + lx;
  int64_t id = tile_off[hilbert_pos(side, tx, ty)] + local;
  order[i] = (int32_t)id;
  inv[id] = (int32_t)i;
}

xct_status make_order(int64_t nx, int64_t ny, int64_t T, int inner, int32_t* order, int32_t* inv,
                      cudaStream_t s) {
  const int64_t ntx = (nx + T - 1) / T, nty = (ny + T - 1) / T;
  int64_t side = 1;
  while (side < std::max(ntx, nty)) side <<= 1;
  if (side * side > (int64_t)1 << 28) {
    set_error("Hilbert tile grid %lld x %lld too large: raise hilbert_tile", (long long)ntx,
              (long long)nty);
    return XCT_ERR_UNSUPPORTED;
  }
  Arena tmp(s);
  int64_t *tsz, *toff;
  XCT_TRY(tmp.get(&tsz, side * side));
  XCT_TRY(tmp.get(&toff, side * side + 1));
  XCT_TRY_CUDA(cudaMemsetAsync(tsz, 0, sizeof(int64_t) * side * side, s));
  tile_sizes_kernel<<<grid_for(ntx * nty, 256), 256, 0, s>>>(nx, ny, T, ntx, nty, side, tsz);
  count_launch();
  XCT_TRY(exclusive_scan_i64(tsz, toff, side * side, s));
  order_kernel<<<grid_for(nx * ny, 256), 256, 0, s>>>(nx, ny, T, side, inner, toff, order, inv);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

// ---------------------------------------------------------------------------
// 2. Siddon trace
// ---------------------------------------------------------------------------

struct Ray {
  double px, py, dx, dy, half, amin, amax, min_seg;
  int n;
};

// Slab clip; false when the ray misses the (closed) grid square or keeps less
// than min_seg of it.
__device__ bool ray_setup(int n, double c, double s, double t, double min_seg, Ray& r) {
  r.n = n;
  r.min_seg = min_seg;
  r.half = dmul(0.5, (double)n);
  r.px = dmul(t, c);
  r.py = dmul(t, s);
  r.dx = -s;
  r.dy = c;
  double amin = -INFINITY, amax = INFINITY;
  if (r.dx != 0.0) {
    double a0 = ddiv(dsub(-r.half, r.px), r.dx), a1 = ddiv(dsub(r.half, r.px), r.dx);
    double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
    if (lo > amin) amin = lo;
    if (hi < amax) amax = hi;
  } else if (!(fabs(r.px) <= r.half)) {
    return false;
  }
  if (r.dy != 0.0) {
    double a0 = ddiv(dsub(-r.half, r.py), r.dy), a1 = ddiv(dsub(r.half, r.py), r.dy);
    double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
    if (lo > amin) amin = lo;
    if (hi < amax) amax = hi;
  } else if (!(fabs(r.py) <= r.half)) {
    return false;
  }
  r.amin = amin;
  r.amax = amax;
  return dsub(amax, amin) >= min_seg;
}

// crossing parameter of interior plane i of an axis (p, d)
__device__ __forceinline__ double plane_alpha(int i, double half, double p, double d) {
  return ddiv(dsub(dsub((double)i, half), p), d);
}

// Crossings of one axis strictly inside (amin, amax), in ascending alpha:
// planes first..last stepping by step (empty when count == 0).  alpha(i) is
// monotone in i, so each bound is found by bisection on the exact predicate.
struct AxisWalk {
  int i, step, left;
};

__device__ AxisWalk axis_walk(const Ray& r, double p, double d) {
  AxisWalk w{0, 1, 0};
  const int n = r.n;
  if (d == 0.0 || n < 2) return w;
  if (d > 0.0) {
    // first i with alpha(i) > amin  (predicate false..true)
    int lo = 1, hi = n;  // hi = none
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (plane_alpha(mid, r.half, p, d) > r.amin) hi = mid; else lo = mid + 1;
    }
    int first = lo;
    // last i with alpha(i) < amax (predicate true..false)
    lo = 0;
    hi = n - 1;  // lo = none
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (plane_alpha(mid, r.half, p, d) < r.amax) lo = mid; else hi = mid - 1;
    }
    int last = lo;
    if (first <= n - 1 && last >= 1 && first <= last) {
      w.i = first;
      w.step = 1;
      w.left = last - first + 1;
    }
  } else {
    // alpha decreasing in i: ascending alpha walks i downwards
    // last i with alpha(i) > amin (predicate true..false)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (plane_alpha(mid, r.half, p, d) > r.amin) lo = mid; else hi = mid - 1;
    }
    int top = lo;
    // first i with alpha(i) < amax (predicate false..true)
    lo = 1;
    hi = n;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (plane_alpha(mid, r.half, p, d) < r.amax) hi = mid; else lo = mid + 1;
    }
    int bottom = lo;
    if (top >= 1 && bottom <= n - 1 && bottom <= top) {
      w.i = top;
      w.step = -1;
      w.left = top - bottom + 1;
    }
  }
  return w;
}

// Walk the merged crossings; sink(pixel, length) for each kept segment.
template <class Sink>
__device__ void trace(const Ray& r, Sink& sink) {
  AxisWalk wx = axis_walk(r, r.px, r.dx);
  AxisWalk wy = axis_walk(r, r.py, r.dy);
  double ax = wx.left ? plane_alpha(wx.i, r.half, r.px, r.dx) : 0.0;
  double ay = wy.left ? plane_alpha(wy.i, r.half, r.py, r.dy) : 0.0;
  double cur = r.amin;
  const int n = r.n;
  while (true) {
    double nxt;
    int which;
    if (wx.left && (!wy.left || ax <= ay)) {
      nxt = ax;
      which = 0;
    } else if (wy.left) {
      nxt = ay;
      which = 1;
    } else {
      nxt = r.amax;
      which = 2;
    }
    double len = dsub(nxt, cur);
    if (len >= r.min_seg) {
      double mid = dmul(dadd(cur, nxt), 0.5);
      double x = dadd(r.px, dmul(mid, r.dx));
      double y = dadd(r.py, dmul(mid, r.dy));
      int ix = (int)floor(dadd(x, r.half));
      int iy = (int)floor(dadd(y, r.half));
      ix = ix < 0 ? 0 : (ix > n - 1 ? n - 1 : ix);
      iy = iy < 0 ? 0 : (iy > n - 1 ? n - 1 : iy);
      sink(iy * n + ix, len);
    }
    cur = nxt;
    if (which == 2) break;
    if (which == 0) {
      wx.i += wx.step;
      if (--wx.left) ax = plane_alpha(wx.i, r.half, r.px, r.dx);
    } else {
      wy.i += wy.step;
      if (--wy.left) ay = plane_alpha(wy.i, r.half, r.py, r.dy);
    }
  }
}

struct GeomDev {
  int n, m, nd;
  double dspace, doff, min_seg;
  const double* cs;  // device [m][2]
};

__device__ __forceinline__ double ray_offset(int j, int nd, double dspace, double doff) {
  return dadd(dmul(dsub((double)j, dmul(0.5, (double)(nd - 1))), dspace), doff);
}

__device__ bool setup_row(const GeomDev& g, int32_t natural_ray, Ray& r) {
  int k = natural_ray / g.nd, j = natural_ray % g.nd;
  return ray_setup(g.n, g.cs[2 * k], g.cs[2 * k + 1], ray_offset(j, g.nd, g.dspace, g.doff),
                   g.min_seg, r);
}

struct CountSink {
  int c = 0;
  __device__ void operator()(int, double) { ++c; }
};

struct FillSink {
  int32_t* col;
  double* val;
  const int32_t* pix_order;
  int64_t pos;
  __device__ void operator()(int pix, double len) {
    col[pos] = pix_order[pix];
    val[pos] = len;
    ++pos;
  }
};

__global__ void siddon_count_kernel(GeomDev g, const int32_t* ray_inv, int64_t nray, int32_t* cnt) {
  int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= nray) return;
  Ray r;
  CountSink sink;
  if (setup_row(g, ray_inv[h], r)) trace(r, sink);
  cnt[h] = sink.c;
}

__global__ void siddon_fill_kernel(GeomDev g, const int32_t* ray_inv, const int32_t* pix_order,
                                   int64_t nray, const int64_t* rowptr, int32_t* col, double* val) {
  int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= nray) return;
  Ray r;
  FillSink sink{col, val, pix_order, rowptr[h]};
  if (setup_row(g, ray_inv[h], r)) trace(r, sink);
}

// Matrix-free projection (no stored A): each thread traces one ray with the
// plan builder's arithmetic and accumulates RN32(length) * x[s][pixel] in
// FP32 for kMfSlices slices per pass, retracing the ray for the next ones.
constexpr int kMfSlices = 8;

struct ProjSink {
  const float* x;      // natural [S][npix]
  int64_t npix;
  int s0, ns;
  float acc[kMfSlices];
  __device__ void operator()(int pix, double len) {
    const float l = (float)len;
#pragma unroll
    for (int k = 0; k < kMfSlices; ++k)
      if (k < ns) acc[k] = fmaf(l, __ldg(x + (size_t)(s0 + k) * npix + pix), acc[k]);
  }
};

__global__ void matfree_project_kernel(GeomDev g, const float* x, float* y, int S, int64_t nray) {
  const int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ray >= nray) return;
  Ray r;
  const bool hit = setup_row(g, (int32_t)ray, r);
  for (int s0 = 0; s0 < S; s0 += kMfSlices) {
    ProjSink sink{x, (int64_t)g.n * g.n, s0, min(kMfSlices, S - s0), {}};
    if (hit) trace(r, sink);
    for (int k = 0; k < sink.ns; ++k) y[(size_t)(s0 + k) * nray + ray] = sink.acc[k];
  }
}

// ---------------------------------------------------------------------------
// 3. transpose
// ---------------------------------------------------------------------------

__global__ void col_count_kernel(const int32_t* col, int64_t nnz, int32_t* ccount) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&ccount[col[e]], 1);
}

__global__ void transpose_fill_kernel(const int64_t* rowptr, const int32_t* col, const double* val,
                                      int64_t nrow, unsigned long long* cursor, int32_t* trow,
                                      double* tval) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    unsigned long long p = atomicAdd(&cursor[col[e]], 1ull);
    trow[p] = (int32_t)r;
    tval[p] = val[e];
  }
}

__global__ void max_count_kernel(const int32_t* c, int64_t n, int32_t* out) {
  int32_t m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, c[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Sort each column's entries by row (bitonic on (row << 32 | position) keys in
// shared memory), making the transpose independent of atomic arrival order.
__global__ void __launch_bounds__(256) column_sort_kernel(const int64_t* colptr, int32_t* trow,
                                                          double* tval, int pow2) {
  extern __shared__ unsigned long long sk[];
  double* sv = reinterpret_cast<double*>(sk + pow2);
  const int64_t c = blockIdx.x;
  const int64_t b = colptr[c];
  const int cnt = (int)(colptr[c + 1] - b);
  if (cnt <= 1) return;
  int p2 = 1;
  while (p2 < cnt) p2 <<= 1;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) {
    if (i < cnt) {
      sk[i] = ((unsigned long long)(uint32_t)trow[b + i] << 32) | (unsigned)i;
      sv[i] = tval[b + i];
    } else {
      sk[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          unsigned long long a = sk[i], bb = sk[l];
          bool up = (i & k) == 0;
          if ((a > bb) == up) {
            sk[i] = bb;
            sk[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    unsigned long long key = sk[i];
    trow[b + i] = (int32_t)(key >> 32);
    tval[b + i] = sv[key & 0xffffffffu];
  }
}

xct_status transpose(const int64_t* rowptr, const int32_t* col, const double* val, int64_t nrow,
                     int64_t ncol, int64_t nnz, int64_t* colptr, int32_t* trow, double* tval,
                     cudaStream_t s) {
  Arena tmp(s);
  int32_t* ccount;
  unsigned long long* cursor;
  int32_t* dmax;
  XCT_TRY(tmp.get(&ccount, ncol));
  XCT_TRY(tmp.get(&cursor, ncol));
  XCT_TRY(tmp.get(&dmax, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(ccount, 0, sizeof(int32_t) * ncol, s));
  XCT_TRY_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
  if (nnz > 0) {
    col_count_kernel<<<grid_for(nnz, 256, 152 * 64), 256, 0, s>>>(col, nnz, ccount);
    count_launch();
  }
  XCT_TRY(exclusive_scan_i32(ccount, colptr, ncol, s));
  XCT_TRY_CUDA(cudaMemcpyAsync(cursor, colptr, sizeof(int64_t) * ncol, cudaMemcpyDeviceToDevice, s));
  if (nnz > 0) {
    transpose_fill_kernel<<<grid_for(nrow, 128), 128, 0, s>>>(rowptr, col, val, nrow, cursor, trow, tval);
    max_count_kernel<<<grid_for(ncol, 256, 1024), 256, 0, s>>>(ccount, ncol, dmax);
    count_launch(2);
    int32_t hmax = 0;
    XCT_TRY_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    XCT_TRY_CUDA(cudaStreamSynchronize(s));
    int p2 = 1;
    while (p2 < hmax) p2 <<= 1;
    size_t smem = (size_t)p2 * 16;
    if (smem > 200 * 1024) {
      set_error("a column holds %d entries; the transpose sort handles at most 8192", hmax);
      return XCT_ERR_UNSUPPORTED;
    }
    if (smem > 48 * 1024)
      XCT_TRY_CUDA(cudaFuncSetAttribute(column_sort_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (hmax > 1) {
      column_sort_kernel<<<(unsigned)ncol, 256, smem, s>>>(colptr, trow, tval, p2);
      count_launch();
    }
  }
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

// ---------------------------------------------------------------------------
// 4. staged kernel layout
// ---------------------------------------------------------------------------

constexpr int kWinBits = 1 << 18;          // columns per footprint window
constexpr int kWinWords = kWinBits / 32;
constexpr int kFpThreads = 512;
constexpr int kStageChunk = 256;           // stages counted per pass

__device__ int64_t block_sum64(int64_t v, int64_t* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

struct CsrView {
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  int64_t nrows, ncols;
};

__device__ void block_col_range(const CsrView& m, int64_t e0, int64_t e1, int32_t* lo_hi) {
  int32_t lo = INT32_MAX, hi = -1;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    int32_t c = m.col[e];
    lo = min(lo, c);
    hi = max(hi, c);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (threadIdx.x == 0) {
    lo_hi[0] = INT32_MAX;
    lo_hi[1] = -1;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&lo_hi[0], lo);
    atomicMax(&lo_hi[1], hi);
  }
  __syncthreads();
}

// Gaps of at most `gap` unreferenced columns between two of a block's
// columns are staged too: a few extra rows per stage join neighbouring runs,
// so a stage needs fewer bulk copies (each costs the TMA unit about 30 ns
// per CTA, whatever its size up to a few KB).  At 512^2 x 768 x 512, gaps
// of up to 4 columns add 7.5% staged rows (A) and cut the runs of a stage
// from 24 to 11; the binary16 products ran 5% / 3.5% faster, FP32 products
// (twice the bytes per staged row) best with gaps of up to 2.
inline int gap_fill_for(xct_dtype storage) { return storage == XCT_F32 ? 2 : 4; }   // < 32

// Mark the block's columns of window [w0, w0 + kWinBits) in the bitmap (and
// the gaps of at most `gap` columns between them inside the window).
__device__ void mark_window(const CsrView& m, int64_t e0, int64_t e1, int64_t w0, int gap,
                            uint32_t* bm) {
  for (int i = threadIdx.x; i < kWinWords; i += blockDim.x) bm[i] = 0;
  __syncthreads();
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    int64_t c = m.col[e] - w0;
    if (c >= 0 && c < kWinBits) atomicOr(&bm[c >> 5], 1u << (c & 31));
  }
  __syncthreads();
  if (gap > 0) {
    constexpr int kPer = kWinWords / kFpThreads;
    static_assert(kWinWords % kFpThreads == 0, "words per thread");
    uint32_t fill[kPer];
    for (int k = 0; k < kPer; ++k) {
      const int i = threadIdx.x * kPer + k;
      const uint64_t lo = i > 0 ? bm[i - 1] : 0u, hi = i + 1 < kWinWords ? bm[i + 1] : 0u;
      const uint32_t mid = bm[i];
      uint32_t f = 0;
      // an empty word lies inside a gap of at least 32 > `gap` columns, and a
      // full word has nothing to fill
      if (mid == 0u || mid == 0xffffffffu) {
        fill[k] = 0u;
        continue;
      }
      for (int j = 0; j < 32; ++j) {
        if ((mid >> j) & 1u) continue;
        // nearest set bits below and above bit j of mid in the 96-bit view
        int dl = 0, dr = 0;
        for (int d = 1; d <= gap; ++d) {
          const int q = 32 + j - d;
          const uint32_t w = q < 32 ? (uint32_t)lo : mid;
          if ((w >> (q & 31)) & 1u) { dl = d; break; }
        }
        for (int d = 1; d <= gap; ++d) {
          const int q = 32 + j + d;
          const uint32_t w = q < 64 ? mid : (uint32_t)hi;
          if ((w >> (q & 31)) & 1u) { dr = d; break; }
        }
        if (dl > 0 && dr > 0 && dl + dr - 1 <= gap) f |= 1u << j;
      }
      fill[k] = f;
    }
    __syncthreads();
    for (int k = 0; k < kPer; ++k) bm[threadIdx.x * kPer + k] |= fill[k];
    __syncthreads();
  }
}

// footprint size (distinct columns) of each block of rows
__global__ void __launch_bounds__(kFpThreads) fp_count_kernel(CsrView m, int gap, int64_t* fp_size) {
  extern __shared__ uint32_t bm[];
  __shared__ int64_t red[kFpThreads / 32];
  __shared__ int32_t lo_hi[2];
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t r1 = min(r0 + kRowsPerBlock, m.nrows);
  const int64_t e0 = m.rowptr[r0], e1 = m.rowptr[r1];
  block_col_range(m, e0, e1, lo_hi);
  int64_t total = 0;
  if (lo_hi[1] >= 0) {
    for (int64_t w0 = (lo_hi[0] / kWinBits) * (int64_t)kWinBits; w0 <= lo_hi[1]; w0 += kWinBits) {
      mark_window(m, e0, e1, w0, gap, bm);
      int64_t c = 0;
      for (int i = threadIdx.x; i < kWinWords; i += blockDim.x) c += __popc(bm[i]);
      total += block_sum64(c, red);
    }
  }
  if (threadIdx.x == 0) fp_size[blockIdx.x] = total;
}

// footprint lists (ascending column) and each entry's footprint position
__global__ void __launch_bounds__(kFpThreads) fp_fill_kernel(CsrView m, int gap, const int64_t* fp_off,
                                                              int32_t* pix, int32_t* epos) {
  extern __shared__ uint32_t bm[];
  int32_t* pre = reinterpret_cast<int32_t*>(bm + kWinWords);
  __shared__ int64_t red[kFpThreads / 32];
  __shared__ int32_t lo_hi[2];
  __shared__ int32_t wtot[kFpThreads / 32];
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t r1 = min(r0 + kRowsPerBlock, m.nrows);
  const int64_t e0 = m.rowptr[r0], e1 = m.rowptr[r1];
  block_col_range(m, e0, e1, lo_hi);
  if (lo_hi[1] < 0) return;
  int64_t base = 0;
  constexpr int kWordsPerThread = kWinWords / kFpThreads;
  for (int64_t w0 = (lo_hi[0] / kWinBits) * (int64_t)kWinBits; w0 <= lo_hi[1]; w0 += kWinBits) {
    mark_window(m, e0, e1, w0, gap, bm);
    // exclusive scan of per-word popcounts: thread t owns words
    // [t*kWordsPerThread, (t+1)*kWordsPerThread)
    int32_t local = 0;
    for (int k = 0; k < kWordsPerThread; ++k) local += __popc(bm[threadIdx.x * kWordsPerThread + k]);
    int32_t inc = local;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    int32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wtot[w];
    int32_t run = woff + inc - local;
    for (int k = 0; k < kWordsPerThread; ++k) {
      int idx = threadIdx.x * kWordsPerThread + k;
      pre[idx] = run;
      run += __popc(bm[idx]);
    }
    __syncthreads();
    // footprint list
    for (int i = threadIdx.x; i < kWinWords; i += blockDim.x) {
      uint32_t bits = bm[i];
      int32_t p = pre[i];
      while (bits) {
        int b = __ffs(bits) - 1;
        bits &= bits - 1;
        pix[fp_off[blockIdx.x] + base + p] = (int32_t)(w0 + i * 32 + b);
        ++p;
      }
    }
    // entry positions
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int64_t c = m.col[e] - w0;
      if (c >= 0 && c < kWinBits) {
        uint32_t word = bm[c >> 5];
        uint32_t below = (c & 31) ? (word & ((1u << (c & 31)) - 1u)) : 0u;
        epos[e] = (int32_t)(base + pre[c >> 5] + __popc(below));
      }
    }
    int64_t wcount = 0;
    for (int w = 0; w < kFpThreads / 32; ++w) wcount += wtot[w];
    base += wcount;
    __syncthreads();
  }
  (void)red;
}

// footprint lists start on 16-byte boundaries: sizes rounded up to 4 ids
__global__ void round4_kernel(const int64_t* in, int32_t n, int64_t* out) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < n) out[b] = (in[b] + 3) & ~(int64_t)3;
}

__global__ void stage_count_kernel(const int64_t* fp_size, int32_t nblocks, int32_t cap,
                                   int64_t* nst) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < nblocks) nst[b] = (fp_size[b] + cap - 1) / cap;
}

__global__ void stage_pix_kernel(const int64_t* blk_stage, const int64_t* fp_off, int32_t nblocks,
                                 int32_t cap, int64_t* stage_pix) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b > nblocks) return;
  if (b == nblocks) {
    stage_pix[blk_stage[nblocks]] = fp_off[nblocks];
    return;
  }
  for (int64_t s = blk_stage[b]; s < blk_stage[b + 1]; ++s)
    stage_pix[s] = fp_off[b] + (s - blk_stage[b]) * cap;
}

// staged rows of each stage (the last stage of a block holds the rest)
__global__ void stage_np_kernel(const int64_t* blk_stage, const int64_t* fp_size, int32_t nblocks,
                                int32_t cap, int32_t* stage_np) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  for (int64_t s = blk_stage[b]; s < blk_stage[b + 1]; ++s)
    stage_np[s] = (int32_t)min((int64_t)cap, fp_size[b] - (s - blk_stage[b]) * cap);
}

// Contiguous runs of each stage's staged rows, for one bulk copy per run:
// pairs (first row id, first position in the stage), then a closing pair
// (-1, rows of the stage) repeated to an even count (16-byte aligned lists).
// One thread per block walks the block's stages.
__global__ void run_count_kernel(const int64_t* blk_stage, const int64_t* fp_off,
                                 const int64_t* fp_size, const int32_t* pix, int32_t nblocks,
                                 int32_t cap, int64_t* nrun, unsigned long long* rmax) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  for (int64_t s = blk_stage[b]; s < blk_stage[b + 1]; ++s) {
    const int64_t k = s - blk_stage[b];
    const int64_t p0 = fp_off[b] + k * cap;
    const int64_t n = min((int64_t)cap, fp_size[b] - k * cap);
    int64_t r = 0;
    for (int64_t i = 0; i < n; ++i)
      if (i == 0 || pix[p0 + i] != pix[p0 + i - 1] + 1) ++r;
    nrun[s] = (r + 2) & ~(int64_t)1;
    atomicMax(rmax, (unsigned long long)nrun[s]);
  }
}

__global__ void run_fill_kernel(const int64_t* blk_stage, const int64_t* fp_off,
                                const int64_t* fp_size, const int32_t* pix, int32_t nblocks,
                                int32_t cap, const int64_t* run_off, int2* runs) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  for (int64_t s = blk_stage[b]; s < blk_stage[b + 1]; ++s) {
    const int64_t k = s - blk_stage[b];
    const int64_t p0 = fp_off[b] + k * cap;
    const int n = (int)min((int64_t)cap, fp_size[b] - k * cap);
    int64_t o = run_off[s];
    for (int i = 0; i < n; ++i)
      if (i == 0 || pix[p0 + i] != pix[p0 + i - 1] + 1) runs[o++] = make_int2(pix[p0 + i], i);
    for (; o < run_off[s + 1]; ++o) runs[o] = make_int2(-1, n);
  }
}

// per (stage, quad): the 4 row counts and the padded slot count (the
// quad's longest row rounded up to `per_row` entries, for each of 4 rows)
__global__ void __launch_bounds__(kRowsPerBlock) seg_count_kernel(CsrView m, const int32_t* epos,
                                                                  const int64_t* blk_stage,
                                                                  int32_t cap, int32_t per_row,
                                                                  Seg* seg, int64_t* slots) {
  __shared__ uint16_t cnt[kRowsPerBlock][kStageChunk + 2];  // counts <= capacity
  const int b = blockIdx.x;
  const int64_t sb = blk_stage[b], ns = blk_stage[b + 1] - sb;
  const int64_t row = (int64_t)b * kRowsPerBlock + threadIdx.x;
  const bool has = row < m.nrows;
  const int64_t e0 = has ? m.rowptr[row] : 0, e1 = has ? m.rowptr[row + 1] : 0;
  for (int64_t s0 = 0; s0 < ns; s0 += kStageChunk) {
    for (int k = 0; k < kStageChunk; ++k) cnt[threadIdx.x][k] = 0;
    for (int64_t e = e0; e < e1; ++e) {
      int64_t st = epos[e] / cap - s0;
      if (st >= 0 && st < kStageChunk) cnt[threadIdx.x][st] = (uint16_t)(cnt[threadIdx.x][st] + 1);
    }
    __syncthreads();
    const int64_t nchunk = min((int64_t)kStageChunk, ns - s0);
    for (int64_t i = threadIdx.x; i < nchunk * kQuads; i += blockDim.x) {
      int64_t st = i / kQuads;
      int q = (int)(i % kQuads);
      Seg sg;
      int32_t mx = 0;
      for (int g = 0; g < 4; ++g) {
        int32_t c = cnt[q * 4 + g][st];
        sg.cnt[g] = (uint16_t)c;
        mx = max(mx, c);
      }
      sg.off = 0;
      int64_t gi = (sb + s0 + st) * kQuads + q;
      seg[gi] = sg;
      slots[gi] = (int64_t)((mx + per_row - 1) / per_row) * per_row * 4;
    }
    __syncthreads();
  }
}

__global__ void seg_off_kernel(Seg* seg, const int64_t* off, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) seg[i].off = off[i];
}

__global__ void stage_ent_kernel(const int64_t* slot_off, int64_t nstages, int64_t* stage_ent,
                                 unsigned long long* emax) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s > nstages) return;
  stage_ent[s] = slot_off[s * kQuads];
  if (s < nstages)
    atomicMax(emax, (unsigned long long)(slot_off[(s + 1) * kQuads] - slot_off[s * kQuads]));
}

// every slot starts as a padding entry: the zero slot (position `zero_slot`)
// with value 0
// one descriptor per stage (see StageDescHead)
__global__ void desc_fill_kernel(const int64_t* stage_ent, const int32_t* stage_np,
                                 const int64_t* stage_run, const int2* runs, const Seg* seg,
                                 int64_t nstages, int64_t run_stride, int64_t desc_bytes,
                                 unsigned char* desc) {
  for (int64_t st = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; st < nstages;
       st += (int64_t)gridDim.x * blockDim.x) {
    unsigned char* d = desc + st * desc_bytes;
    StageDescHead h;
    h.e0 = stage_ent[st];
    h.slots = (uint32_t)(stage_ent[st + 1] - stage_ent[st]);
    h.np = (uint16_t)stage_np[st];
    const int64_t r0 = stage_run[st], nr = stage_run[st + 1] - r0;
    h.nr = (uint16_t)nr;
    *reinterpret_cast<StageDescHead*>(d) = h;
    uint4* sd = reinterpret_cast<uint4*>(d + sizeof(StageDescHead));
    const uint4* ss = reinterpret_cast<const uint4*>(seg + st * kQuads);
    for (int q = 0; q < kQuads; ++q) sd[q] = ss[q];
    int2* rd = reinterpret_cast<int2*>(d + sizeof(StageDescHead) + kQuads * 16);
    for (int64_t k = 0; k < run_stride; ++k)
      rd[k] = k < nr ? runs[r0 + k] : make_int2(-1, (int)h.np);
  }
}

template <int EB>
__global__ void pad_fill_kernel(void* ent, int64_t nslots, uint32_t zero_slot, uint32_t unit) {
  const uint32_t off = zero_slot * unit;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nslots;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (EB == 4)
      static_cast<uint32_t*>(ent)[i] = off << 16;
    else
      static_cast<unsigned long long*>(ent)[i] = off;
  }
}

template <int KIND>  // 0: f32, 1: f16 (x 2^15), 2: bf16
__device__ __forceinline__ void pack_entry(void* ent, int64_t slot, uint32_t local, double v,
                                           uint32_t unit) {
  const uint32_t off = local * unit;
  if (KIND == 0) {
    unsigned long long w = (unsigned long long)off |
                           ((unsigned long long)__float_as_uint(__double2float_rn(v)) << 32);
    static_cast<unsigned long long*>(ent)[slot] = w;
  } else if (KIND == 1) {
    unsigned short h = __half_as_ushort(__double2half(dmul(v, 32768.0)));
    static_cast<uint32_t*>(ent)[slot] = (off << 16) | h;
  } else {
    unsigned short h = __bfloat16_as_ushort(__double2bfloat16(v));
    static_cast<uint32_t*>(ent)[slot] = (off << 16) | h;
  }
}

template <int KIND>
__global__ void __launch_bounds__(kRowsPerBlock) fill_entries_kernel(CsrView m, const int32_t* epos,
                                                                     const int64_t* blk_stage,
                                                                     int32_t cap, const Seg* seg,
                                                                     void* ent, uint32_t unit) {
  __shared__ uint16_t cnt[kRowsPerBlock][kStageChunk + 2];  // counts <= capacity
  const int b = blockIdx.x;
  const int64_t sb = blk_stage[b], ns = blk_stage[b + 1] - sb;
  const int64_t row = (int64_t)b * kRowsPerBlock + threadIdx.x;
  if (row >= m.nrows) return;
  const int q = threadIdx.x / 4, g = threadIdx.x % 4;
  const int64_t e0 = m.rowptr[row], e1 = m.rowptr[row + 1];
  for (int64_t s0 = 0; s0 < ns; s0 += kStageChunk) {
    for (int k = 0; k < kStageChunk; ++k) cnt[threadIdx.x][k] = 0;
    for (int64_t e = e0; e < e1; ++e) {
      int32_t p = epos[e];
      int64_t st = p / cap - s0;
      if (st < 0 || st >= kStageChunk) continue;
      int32_t k = cnt[threadIdx.x][st];
      cnt[threadIdx.x][st] = (uint16_t)(k + 1);
      int64_t slot = seg[(sb + s0 + st) * kQuads + q].off + (k >> 2) * 16 + g * 4 + (k & 3);
      pack_entry<KIND>(ent, slot, (uint32_t)(p % cap), m.val[e], unit);
    }
  }
}

// Entry order of a wide-stage layout (16-byte staged rows, 16-bit entries).
// The product kernel's four lanes of a row read, at one time step, slot q of
// chunks 4i .. 4i + 3 (lane e takes chunk 4i + e), and the lanes of the two
// rows g = 2h, 2h + 1 of a quad issue their loads together (one phase of 8
// lanes of a 16-byte load).
//  - Placement: a quad's chunks lie in groups of 4 per row, one group of all
//    4 rows after the other (chunk c of row g at 16-byte chunk
//    (c / 4) * 16 + g * 4 + c % 4; the segment holds the quad's longest row
//    rounded up to 16 entries for each row), so the 8 lanes of a phase read
//    128 contiguous bytes of entries.
//  - Order: staged row j lies in shared-memory bank group j mod 8, so two of
//    a phase's 8 reads of staged rows conflict when their rows differ and
//    share the group.  The order of a row's entries is free (the row's sum
//    is the same up to the rounding of its FP32 accumulation), so this pass
//    takes each half quad's entries one time step at a time, giving the 8
//    reads distinct groups where the remaining entries allow: for each lane
//    an entry of the free group with the most entries left in its row, else
//    a padding entry (the zero slot; several of them in a phase read one
//    address), else an entry of the row's largest group.
// `src` is a copy of the entries in the CSR-order placement of
// fill_entries_kernel, `ent` starts as padding; one thread per half quad.
__global__ void wide_order_kernel(const uint32_t* src, uint32_t* ent, const Seg* seg,
                                  int64_t nhalf, uint32_t zero_entry) {
  const int zg = (int)((zero_entry >> 20) & 7u);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nhalf;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Seg sg = seg[t >> 1];
    const int h = (int)(t & 1);
    int cnt[2], nch[2], pads[2];
    int left[2][8], scan[2][8];
    for (int r = 0; r < 2; ++r) {
      cnt[r] = sg.cnt[2 * h + r];
      nch[r] = (cnt[r] + 3) >> 2;
      pads[r] = 4 * nch[r] - cnt[r];
      for (int b = 0; b < 8; ++b) left[r][b] = 0, scan[r][b] = 0;
    }
    auto slot = [&](int r, int k) { return sg.off + (k >> 2) * 16 + (2 * h + r) * 4 + (k & 3); };
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < cnt[r]; ++k) ++left[r][(src[slot(r, k)] >> 20) & 7u];
    const int nmax = nch[0] > nch[1] ? nch[0] : nch[1];
    for (int i = 0; 4 * i < nmax; ++i)
      for (int q = 0; q < 4; ++q) {
        uint32_t used = 0;     // groups taken by matrix entries at this step
        bool pad_here = false;
        for (int e = 0; e < 4; ++e)
          for (int r = 0; r < 2; ++r) {
            const int c = 4 * i + e;
            if (c >= nch[r]) continue;
            int best = -1;
            for (int b = 0; b < 8; ++b)
              if (left[r][b] > 0 && !((used >> b) & 1u) && !(pad_here && b == zg) &&
                  (best < 0 || left[r][b] > left[r][best]))
                best = b;
            uint32_t v;
            if (best < 0 && pads[r] > 0 && !((used >> zg) & 1u)) {
              v = zero_entry;
              --pads[r];
              pad_here = true;
            } else {
              if (best < 0)
                for (int b = 0; b < 8; ++b)
                  if (left[r][b] > 0 && (best < 0 || left[r][b] > left[r][best])) best = b;
              if (best < 0) {   // only padding left in this row
                v = zero_entry;
                --pads[r];
                pad_here = true;
              } else {
                int k = scan[r][best];   // an entry of group `best` lies at or after k
                while (k < cnt[r] - 1 && ((src[slot(r, k)] >> 20) & 7u) != (uint32_t)best) ++k;
                v = src[slot(r, k)];
                scan[r][best] = k + 1;
                --left[r][best];
                used |= 1u << best;
              }
            }
            const int g = 2 * h + r;
            ent[sg.off + ((int64_t)i * 16 + g * 4 + e) * 4 + q] = v;
          }
      }
  }
}

// Entry order of a 280-row layout (128-byte staged-row offsets) for the
// narrower slice tiles that read it (plans built with XCT_PLAN_NARROW_TILES).  With 32-byte rows (16 slices) the
// lanes of a quad's 4 rows read their k-th entries together (one phase of a
// 16-byte load), staged row j lying in the 8-bank group j mod 4; with
// 64-byte rows (32 slices) rows 2h and 2h + 1 share a phase, row j in bank
// half j mod 2.  So at every entry index the plan gives the quad's rows
// distinct residues mod 4 where the counts allow, rows 2h and 2h + 1 of
// different parity where it can: for each row, the free residue with the
// most entries left (for the second row of a pair, one of the other parity
// first).  The order of a row's entries is free (its sum changes only by
// FP32 rounding); padding stays at the end of each row.  `src` is a copy of
// the entries in CSR order; one thread per (stage, quad).
__global__ void quad_order_kernel(const uint32_t* src, uint32_t* ent, const Seg* seg, int64_t nquads) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nquads;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Seg sg = seg[t];
    int cnt[4], left[4][4], scan[4][4];
    int kmax = 0;
    for (int g = 0; g < 4; ++g) {
      cnt[g] = sg.cnt[g];
      kmax = kmax > cnt[g] ? kmax : cnt[g];
      for (int b = 0; b < 4; ++b) left[g][b] = 0, scan[g][b] = 0;
    }
    auto slot = [&](int g, int k) { return sg.off + (k >> 2) * 16 + g * 4 + (k & 3); };
    auto group = [&](uint32_t e) { return (int)((e >> 23) & 3u); };   // (offset / 128) mod 4
    for (int g = 0; g < 4; ++g)
      for (int k = 0; k < cnt[g]; ++k) ++left[g][group(src[slot(g, k)])];
    for (int k = 0; k < kmax; ++k) {
      uint32_t used = 0;
      int pick[4] = {-1, -1, -1, -1};
      for (int g = 0; g < 4; ++g) {
        if (k >= cnt[g]) continue;
        const int partner = (g & 1) ? pick[g - 1] : -1;
        int best = -1;
        for (int pass = 0; pass < 3 && best < 0; ++pass)
          for (int b = 0; b < 4; ++b) {
            if (left[g][b] == 0) continue;
            if (pass < 2 && ((used >> b) & 1u)) continue;
            if (pass == 0 && partner >= 0 && (b & 1) == (partner & 1)) continue;
            if (best < 0 || left[g][b] > left[g][best]) best = b;
          }
        int j = scan[g][best];   // an entry of group `best` lies at or after j
        while (j < cnt[g] - 1 && group(src[slot(g, j)]) != best) ++j;
        ent[slot(g, k)] = src[slot(g, j)];
        scan[g][best] = j + 1;
        --left[g][best];
        used |= 1u << best;
        pick[g] = best;
      }
    }
  }
}

xct_status build_layout(const CsrView& m, int64_t nnz, xct_dtype storage, int32_t cap, Layout& L,
                        Arena& keep, cudaStream_t s, int gap = -1,
                        int32_t unit = kEntryRowBytes, bool quad_order = false) {
  if (gap < 0) gap = gap_fill_for(storage);
  L.nrows = m.nrows;
  L.ncols = m.ncols;
  L.cap = cap;
  L.unit = unit;
  L.ebytes = storage == XCT_F32 ? 8 : 4;
  L.nblocks = (int32_t)((m.nrows + kRowsPerBlock - 1) / kRowsPerBlock);
  const int32_t nb = L.nblocks;
  Arena tmp(s);
  int64_t *fp_size, *fp_pad, *fp_off, *nst;
  int32_t* epos;
  XCT_TRY(tmp.get(&fp_size, nb));
  XCT_TRY(tmp.get(&fp_pad, nb));
  XCT_TRY(tmp.get(&fp_off, nb + 1));
  XCT_TRY(tmp.get(&nst, nb));
  XCT_TRY(tmp.get(&epos, nnz));
  const size_t bm_smem = (size_t)kWinWords * 4;
  const size_t fill_smem = (size_t)kWinWords * 8;
  XCT_TRY_CUDA(cudaFuncSetAttribute(fp_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bm_smem));
  XCT_TRY_CUDA(cudaFuncSetAttribute(fp_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)fill_smem));
  if (nb > 0) {
    fp_count_kernel<<<nb, kFpThreads, bm_smem, s>>>(m, gap, fp_size);
    count_launch();
  }
  if (nb > 0) {
    round4_kernel<<<grid_for(nb, 256), 256, 0, s>>>(fp_size, nb, fp_pad);
    count_launch();
  }
  XCT_TRY(exclusive_scan_i64(fp_pad, fp_off, nb, s));
  int64_t total_fp = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&total_fp, fp_off + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  L.footprint = total_fp;
  Arena own(s);
  XCT_TRY(own.get(&L.pix, total_fp + 4));   // padded lists, +4 for rounded copies
  XCT_TRY_CUDA(cudaMemsetAsync(L.pix, 0, sizeof(int32_t) * (total_fp + 4), s));
  XCT_TRY(own.get(&L.blk_stage, nb + 1));
  if (nb > 0) {
    fp_fill_kernel<<<nb, kFpThreads, fill_smem, s>>>(m, gap, fp_off, L.pix, epos);
    stage_count_kernel<<<grid_for(nb, 256), 256, 0, s>>>(fp_size, nb, cap, nst);
    count_launch(2);
  }
  XCT_TRY(exclusive_scan_i64(nst, L.blk_stage, nb, s));
  XCT_TRY_CUDA(cudaMemcpyAsync(&L.nstages, L.blk_stage + nb, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  XCT_TRY(own.get(&L.stage_pix, L.nstages + 1));
  XCT_TRY(own.get(&L.seg, L.nstages * kQuads));
  int64_t *slots, *slot_off;
  XCT_TRY(tmp.get(&slots, L.nstages * kQuads));
  XCT_TRY(tmp.get(&slot_off, L.nstages * kQuads + 1));
  stage_pix_kernel<<<grid_for(nb + 1, 256), 256, 0, s>>>(L.blk_stage, fp_off, nb, cap, L.stage_pix);
  count_launch();
  XCT_TRY(own.get(&L.stage_np, L.nstages));
  if (nb > 0) {
    stage_np_kernel<<<grid_for(nb, 256), 256, 0, s>>>(L.blk_stage, fp_size, nb, cap, L.stage_np);
    count_launch();
  }
  {
    int64_t* nrun;
    unsigned long long* rmax;
    XCT_TRY(tmp.get(&nrun, L.nstages));
    XCT_TRY(tmp.get(&rmax, 1));
    XCT_TRY(own.get(&L.stage_run, L.nstages + 1));
    XCT_TRY_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s));
    if (nb > 0) {
      run_count_kernel<<<grid_for(nb, 128), 128, 0, s>>>(L.blk_stage, fp_off, fp_size, L.pix, nb, cap,
                                                         nrun, rmax);
      count_launch();
    }
    XCT_TRY(exclusive_scan_i64(nrun, L.stage_run, L.nstages, s));
    int64_t nruns = 0;
    unsigned long long rmax_h = 0;
    XCT_TRY_CUDA(cudaMemcpyAsync(&nruns, L.stage_run + L.nstages, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    XCT_TRY_CUDA(cudaMemcpyAsync(&rmax_h, rmax, sizeof(rmax_h), cudaMemcpyDeviceToHost, s));
    XCT_TRY_CUDA(cudaStreamSynchronize(s));
    L.nruns = nruns;
    L.run_max = (int64_t)rmax_h;
    XCT_TRY(own.get(&L.runs, nruns));
    if (nb > 0) {
      run_fill_kernel<<<grid_for(nb, 128), 128, 0, s>>>(L.blk_stage, fp_off, fp_size, L.pix, nb, cap,
                                                        L.stage_run, L.runs);
      count_launch();
    }
  }
  if (nb > 0) {
    // wide-stage layouts: groups of 4 chunks per row (see wide_order_kernel)
    seg_count_kernel<<<nb, kRowsPerBlock, 0, s>>>(m, epos, L.blk_stage, cap,
                                                  unit == kWideRowBytes ? 16 : 4, L.seg, slots);
    count_launch();
  }
  XCT_TRY(exclusive_scan_i64(slots, slot_off, L.nstages * kQuads, s));
  if (L.nstages > 0) {
    seg_off_kernel<<<grid_for(L.nstages * kQuads, 256), 256, 0, s>>>(L.seg, slot_off,
                                                                    L.nstages * kQuads);
    count_launch();
  }
  XCT_TRY_CUDA(cudaMemcpyAsync(&L.nslots, slot_off + L.nstages * kQuads, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
  XCT_TRY(own.get(&L.stage_ent, L.nstages + 1));
  unsigned long long* emax;
  XCT_TRY(tmp.get(&emax, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(emax, 0, sizeof(unsigned long long), s));
  stage_ent_kernel<<<grid_for(L.nstages + 1, 256), 256, 0, s>>>(slot_off, L.nstages, L.stage_ent, emax);
  count_launch();
  unsigned long long emax_h = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&emax_h, emax, sizeof(emax_h), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  L.emax_slots = (int64_t)emax_h;
  if (L.ebytes == 8) {
    unsigned long long* e;
    XCT_TRY(own.get(&e, L.nslots));
    L.ent = e;
    pad_fill_kernel<8><<<grid_for(L.nslots, 256, 152 * 32), 256, 0, s>>>(L.ent, L.nslots, (uint32_t)cap,
                                                                         (uint32_t)unit);
  } else {
    uint32_t* e;
    XCT_TRY(own.get(&e, L.nslots));
    L.ent = e;
    pad_fill_kernel<4><<<grid_for(L.nslots, 256, 152 * 32), 256, 0, s>>>(L.ent, L.nslots, (uint32_t)cap,
                                                                         (uint32_t)unit);
  }
  count_launch();
  if (nb > 0) {
    if (storage == XCT_F32)
      fill_entries_kernel<0><<<nb, kRowsPerBlock, 0, s>>>(m, epos, L.blk_stage, cap, L.seg, L.ent,
                                                            (uint32_t)unit);
    else if (half_values(storage))
      fill_entries_kernel<1><<<nb, kRowsPerBlock, 0, s>>>(m, epos, L.blk_stage, cap, L.seg, L.ent,
                                                            (uint32_t)unit);
    else
      fill_entries_kernel<2><<<nb, kRowsPerBlock, 0, s>>>(m, epos, L.blk_stage, cap, L.seg, L.ent,
                                                            (uint32_t)unit);
    count_launch();
  }
  if (unit == kWideRowBytes && L.ebytes == 4 && L.nslots > 0) {
    uint32_t* src;
    XCT_TRY(tmp.get(&src, L.nslots));
    XCT_TRY_CUDA(cudaMemcpyAsync(src, L.ent, sizeof(uint32_t) * L.nslots, cudaMemcpyDeviceToDevice, s));
    pad_fill_kernel<4><<<grid_for(L.nslots, 256, 152 * 32), 256, 0, s>>>(L.ent, L.nslots, (uint32_t)cap,
                                                                         (uint32_t)unit);
    count_launch();
    const int64_t nhalf = L.nstages * kQuads * 2;
    wide_order_kernel<<<grid_for(nhalf, 128), 128, 0, s>>>(src, static_cast<uint32_t*>(L.ent), L.seg,
                                                           nhalf, ((uint32_t)cap * unit) << 16);
    count_launch();
  }
  if (quad_order && unit == kEntryRowBytes && L.ebytes == 4 && L.nslots > 0) {
    uint32_t* src;
    XCT_TRY(tmp.get(&src, L.nslots));
    XCT_TRY_CUDA(cudaMemcpyAsync(src, L.ent, sizeof(uint32_t) * L.nslots, cudaMemcpyDeviceToDevice, s));
    const int64_t nq = L.nstages * kQuads;
    quad_order_kernel<<<grid_for(nq, 128), 128, 0, s>>>(src, static_cast<uint32_t*>(L.ent), L.seg, nq);
    count_launch();
  }
  // stage descriptors: run lists padded to an even count of at least 2
  {
    const int64_t stride = L.run_max < 2 ? 2 : (L.run_max + 1) & ~(int64_t)1;
    L.desc_bytes = stage_desc_bytes(stride);
    XCT_TRY(own.get(&L.desc, (size_t)(L.nstages > 0 ? L.nstages : 1) * L.desc_bytes));
    if (L.nstages > 0) {
      desc_fill_kernel<<<grid_for(L.nstages, 128, 152 * 16), 128, 0, s>>>(
          L.stage_ent, L.stage_np, L.stage_run, L.runs, L.seg, L.nstages, stride, L.desc_bytes,
          L.desc);
      count_launch();
    }
  }
  XCT_TRY_CUDA(cudaGetLastError());
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  L.bytes = (int64_t)L.nslots * L.ebytes + L.nstages * kQuads * (int64_t)sizeof(Seg) +
            (L.nstages + 1) * 24 + L.nstages * 4 + (int64_t)(nb + 1) * 8 + total_fp * 4 +
            L.nruns * 8 + L.nstages * L.desc_bytes;
  own.move_to(keep);
  return XCT_OK;
}

// Paired layout of a 280-row layout of 16-bit values (XCT_PLAN_PAIRED_ROWS;
// the slot placement is described with kPairUA in xct_internal.cuh).  The
// positions of a row's entries in a stage are distinct (a ray crosses a pixel
// once), so the columns two rows share are the intersection of two position
// bitmaps (at most kMaxStageCap + 1 positions).  One thread per (stage,
// quad); `src` is the plain layout's entries (row g's k-th entry of the
// segment at off + (k / 4) * 16 + g * 4 + k % 4, any order within the row).
constexpr int kPairBmWords = (kMaxStageCap + 1 + 31) / 32;

__device__ __forceinline__ int pair_pos(uint32_t e) { return (int)((e >> 16) / (uint32_t)kEntryRowBytes); }

__device__ __forceinline__ int64_t pair_src_slot(const Seg& sg, int g, int k) {
  return sg.off + (int64_t)(k >> 2) * 16 + g * 4 + (k & 3);
}

__device__ void pair_bitmaps(const uint32_t* src, const Seg& sg, int p, uint32_t* b0, uint32_t* b1) {
  for (int i = 0; i < kPairBmWords; ++i) b0[i] = 0u, b1[i] = 0u;
  for (int k = 0; k < sg.cnt[2 * p]; ++k) {
    const int q = pair_pos(src[pair_src_slot(sg, 2 * p, k)]);
    b0[q >> 5] |= 1u << (q & 31);
  }
  for (int k = 0; k < sg.cnt[2 * p + 1]; ++k) {
    const int q = pair_pos(src[pair_src_slot(sg, 2 * p + 1, k)]);
    b1[q >> 5] |= 1u << (q & 31);
  }
}

__host__ __device__ inline int pair_groups(int chunks, int per) { return (chunks + per - 1) / per; }

__global__ void pair_count_kernel(const uint32_t* src, const Seg* seg, int64_t nquads, Seg* pseg,
                                  int64_t* slots, unsigned long long* gathers) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nquads;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Seg sg = seg[t];
    Seg ps;
    ps.off = 0;
    unsigned long long uni = 0;   // distinct columns of the pairs: staged-row reads
    for (int p = 0; p < 2; ++p) {
      uint32_t b0[kPairBmWords], b1[kPairBmWords];
      pair_bitmaps(src, sg, p, b0, b1);
      int ns = 0;
      for (int i = 0; i < kPairBmWords; ++i) ns += __popc(b0[i] & b1[i]);
      const int c0 = sg.cnt[2 * p], c1 = sg.cnt[2 * p + 1];
      const int nx = (c0 > c1 ? c0 : c1) - ns;
      uni += (unsigned long long)(c0 + c1 - ns);
      ps.cnt[2 * p] = (uint16_t)((ns + 1) >> 1);
      ps.cnt[2 * p + 1] = (uint16_t)((nx + 1) >> 1);
    }
    const int ga = pair_groups(ps.cnt[0] > ps.cnt[2] ? ps.cnt[0] : ps.cnt[2], kPairUA);
    const int gb = pair_groups(ps.cnt[1] > ps.cnt[3] ? ps.cnt[1] : ps.cnt[3], kPairUB);
    pseg[t] = ps;
    slots[t] = (int64_t)ga * 4 * kPairUA + (int64_t)gb * 4 * kPairUB;
    if (uni) atomicAdd(gathers, uni);
  }
}

// `dst` starts as padding (both halves of every slot: the zero slot, value
// 0); `bad` counts segments whose lists disagree with the counted sizes
// (none for a traced matrix)
__global__ void pair_fill_kernel(const uint32_t* src, const Seg* seg, const Seg* pseg, int64_t nquads,
                                 uint32_t* dst, unsigned int* bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nquads;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Seg sg = seg[t], ps = pseg[t];
    const int ga = pair_groups(ps.cnt[0] > ps.cnt[2] ? ps.cnt[0] : ps.cnt[2], kPairUA);
    const int64_t reg_a = ps.off, reg_b = ps.off + (int64_t)ga * 4 * kPairUA;
    for (int p = 0; p < 2; ++p) {
      uint32_t b0[kPairBmWords], b1[kPairBmWords];
      pair_bitmaps(src, sg, p, b0, b1);
      const int c0 = sg.cnt[2 * p], c1 = sg.cnt[2 * p + 1];
      const int ns_cap = 2 * ps.cnt[2 * p], nx_cap = 2 * ps.cnt[2 * p + 1];
      // slot of index i among a pair's shared (split) slots: chunk i / 2,
      // lane i % 2
      auto sa = [&](int i) {
        const int c = i >> 1, e = i & 1;
        return reg_a + (int64_t)(c / kPairUA) * 4 * kPairUA + (2 * p + e) * kPairUA + c % kPairUA;
      };
      auto sb = [&](int i) {
        const int c = i >> 1, e = i & 1;
        return reg_b + (int64_t)(c / kPairUB) * 4 * kPairUB + (2 * p + e) * kPairUB + c % kPairUB;
      };
      int ns = 0, n0 = 0, n1 = 0;
      for (int k = 0; k < c0; ++k) {
        const uint32_t e = src[pair_src_slot(sg, 2 * p, k)];
        const int q = pair_pos(e);
        if ((b1[q >> 5] >> (q & 31)) & 1u) {
          uint32_t f = 0u;
          for (int j = 0; j < c1; ++j) {
            const uint32_t h = src[pair_src_slot(sg, 2 * p + 1, j)];
            if ((h >> 16) == (e >> 16)) { f = h; break; }
          }
          if (ns < ns_cap) {
            dst[2 * sa(ns)] = e;
            dst[2 * sa(ns) + 1] = f;
          } else {
            atomicAdd(bad, 1u);
          }
          ++ns;
        } else {
          if (n0 < nx_cap) dst[2 * sb(n0)] = e;
          else atomicAdd(bad, 1u);
          ++n0;
        }
      }
      for (int k = 0; k < c1; ++k) {
        const uint32_t e = src[pair_src_slot(sg, 2 * p + 1, k)];
        const int q = pair_pos(e);
        if ((b0[q >> 5] >> (q & 31)) & 1u) continue;
        if (n1 < nx_cap) dst[2 * sb(n1) + 1] = e;
        else atomicAdd(bad, 1u);
        ++n1;
      }
    }
  }
}

__global__ void pair_pad_kernel(uint32_t* dst, int64_t n, uint32_t zero_entry) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = zero_entry;
}

// The paired layout P of a built 280-row layout L of 16-bit values: the
// stages, footprints, run lists and stage capacity are L's (shared, not
// copied); segments, slots and stage descriptors are P's own.
xct_status build_paired_layout(const Layout& L, Layout& P, Arena& keep, cudaStream_t s) {
  if (L.ebytes != 4 || L.unit != kEntryRowBytes || L.cap > kMaxStageCap) {
    set_error("paired layout: needs a 280-row layout of 16-bit values");
    return XCT_ERR_INVALID;
  }
  P = Layout{};
  P.nrows = L.nrows;
  P.ncols = L.ncols;
  P.nblocks = L.nblocks;
  P.cap = L.cap;
  P.ebytes = 8;
  P.nstages = L.nstages;
  P.footprint = L.footprint;
  P.blk_stage = L.blk_stage;
  P.stage_pix = L.stage_pix;
  P.stage_np = L.stage_np;
  P.pix = L.pix;
  P.stage_run = L.stage_run;
  P.runs = L.runs;
  P.nruns = L.nruns;
  P.run_max = L.run_max;
  P.unit = kEntryRowBytes;
  P.pair = true;
  const int64_t nq = L.nstages * kQuads;
  Arena tmp(s), own(s);
  int64_t *slots, *slot_off;
  unsigned int* bad;
  unsigned long long *emax, *gath;
  XCT_TRY(own.get(&P.seg, nq > 0 ? nq : 1));
  XCT_TRY(tmp.get(&gath, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(gath, 0, sizeof(unsigned long long), s));
  XCT_TRY(tmp.get(&slots, nq > 0 ? nq : 1));
  XCT_TRY(tmp.get(&slot_off, nq + 1));
  XCT_TRY(tmp.get(&bad, 1));
  XCT_TRY(tmp.get(&emax, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
  XCT_TRY_CUDA(cudaMemsetAsync(emax, 0, sizeof(unsigned long long), s));
  const uint32_t* src = static_cast<const uint32_t*>(L.ent);
  if (nq > 0) {
    pair_count_kernel<<<grid_for(nq, 128, 152 * 64), 128, 0, s>>>(src, L.seg, nq, P.seg, slots, gath);
    count_launch();
  }
  XCT_TRY(exclusive_scan_i64(slots, slot_off, nq, s));
  if (nq > 0) {
    seg_off_kernel<<<grid_for(nq, 256), 256, 0, s>>>(P.seg, slot_off, nq);
    count_launch();
  }
  XCT_TRY_CUDA(cudaMemcpyAsync(&P.nslots, slot_off + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XCT_TRY(own.get(&P.stage_ent, P.nstages + 1));
  stage_ent_kernel<<<grid_for(P.nstages + 1, 256), 256, 0, s>>>(slot_off, P.nstages, P.stage_ent, emax);
  count_launch();
  unsigned long long emax_h = 0, gath_h = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&emax_h, emax, sizeof(emax_h), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaMemcpyAsync(&gath_h, gath, sizeof(gath_h), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  P.emax_slots = (int64_t)emax_h;
  P.gathers = (int64_t)gath_h;
  uint2* ent;
  XCT_TRY(own.get(&ent, P.nslots > 0 ? P.nslots : 1));
  P.ent = ent;
  if (P.nslots > 0) {
    pair_pad_kernel<<<grid_for(2 * P.nslots, 256, 152 * 32), 256, 0, s>>>(
        reinterpret_cast<uint32_t*>(ent), 2 * P.nslots, ((uint32_t)L.cap * kEntryRowBytes) << 16);
    count_launch();
  }
  if (nq > 0) {
    pair_fill_kernel<<<grid_for(nq, 128, 152 * 64), 128, 0, s>>>(src, L.seg, P.seg, nq,
                                                                reinterpret_cast<uint32_t*>(ent), bad);
    count_launch();
  }
  {
    const int64_t stride = L.run_max < 2 ? 2 : (L.run_max + 1) & ~(int64_t)1;
    P.desc_bytes = stage_desc_bytes(stride);
    XCT_TRY(own.get(&P.desc, (size_t)(P.nstages > 0 ? P.nstages : 1) * P.desc_bytes));
    if (P.nstages > 0) {
      desc_fill_kernel<<<grid_for(P.nstages, 128, 152 * 16), 128, 0, s>>>(
          P.stage_ent, P.stage_np, P.stage_run, P.runs, P.seg, P.nstages, stride, P.desc_bytes, P.desc);
      count_launch();
    }
  }
  unsigned int bad_h = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(bad_h), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaGetLastError());
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  if (bad_h != 0) {
    set_error("paired layout: %u entries outside their counted lists", bad_h);
    return XCT_ERR_CUDA;
  }
  P.bytes = P.nslots * 8 + nq * (int64_t)sizeof(Seg) + (P.nstages + 1) * 8 + P.nstages * P.desc_bytes;
  own.move_to(keep);
  return XCT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------

// Time one product on layout L at the widest slice tile of the plan's
// storage (inputs zero: the work does not depend on the values), after one
// warm-up; the mean of two launches in milliseconds.
xct_status time_product(const Layout& L, Plan& p, cudaStream_t s, double* ms_out) {
  const int st = pick_slices_per_tile(p.storage, 64);
  Arena ar(s);
  float *xi, *yi;
  uint16_t* h = nullptr;
  uint32_t* mx;
  double* dot;
  int* work;
  XCT_TRY(ar.get(&xi, (size_t)L.ncols * st));
  XCT_TRY(ar.get(&yi, (size_t)L.nrows * st));
  if (stages16(p.storage)) XCT_TRY(ar.get(&h, (size_t)L.ncols * st));
  XCT_TRY(ar.get(&mx, (size_t)st));
  XCT_TRY(ar.get(&dot, (size_t)st * std::max(L.nblocks, 1)));
  XCT_TRY(ar.get(&work, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(xi, 0, sizeof(float) * L.ncols * st, s));
  XCT_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(uint32_t) * st, s));
  SpmmArgs a{&L, xi, yi, st, 1, p.storage, p.mat_scale_exp, mx, dot, h, work, p.err};
  cudaEvent_t e0, e1;
  XCT_TRY_CUDA(cudaEventCreate(&e0));
  XCT_TRY_CUDA(cudaEventCreate(&e1));
  xct_status r = spmm(a, s);
  if (r == XCT_OK) cudaEventRecord(e0, s);
  for (int k = 0; k < 2 && r == XCT_OK; ++k) r = spmm(a, s);
  if (r == XCT_OK) cudaEventRecord(e1, s);
  float ms = 0.0f;
  cudaError_t ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess && r == XCT_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  XCT_TRY(r);
  if (ce != cudaSuccess) {
    set_error("stage capacity timing failed: %s", cudaGetErrorString(ce));
    return XCT_ERR_CUDA;
  }
  *ms_out = ms / 2.0;
  return XCT_OK;
}

// Matrix-free back projection, pixel-driven: x[s][pixel] = sum over the rays
// through the pixel, in ascending ray id, of RN32(length) * y[s][ray] in
// FP32.  A ray's length in a pixel is its traced segment there, found
// without tracing: the ray's crossings of the pixel's four boundary planes
// (the same plane_alpha doubles the trace merges; planes 0 and n give the
// slab clip's doubles) and the ray's clip interval bound it, no other
// crossing lies strictly inside, and the trace keeps the segment when it is
// at least min_seg long, assigning it to the pixel of its midpoint.  So the
// lengths equal the stored matrix's values bit for bit (min_seg > 0; with
// min_seg = 0 the trace also keeps the slivers, below 1e-14, that rounding
// leaves between crossings which coincide in real arithmetic).
__global__ void matfree_ray_setup_kernel(GeomDev g, int64_t nray, double4* rs) {
  const int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ray >= nray) return;
  Ray r;
  // amin > amax marks a ray that is not traced (it misses the grid or keeps
  // less than min_seg of it)
  rs[ray] = setup_row(g, (int32_t)ray, r) ? make_double4(r.px, r.py, r.amin, r.amax)
                                          : make_double4(0.0, 0.0, 1.0, 0.0);
}

// the alpha interval of the ray inside pixel column (row) i of one axis;
// false when the axis is parallel to the ray and the line is outside it
__device__ __forceinline__ bool pixel_axis(int i, int n, double half, double p, double d,
                                           double& lo, double& hi) {
  if (d != 0.0) {
    const double a0 = plane_alpha(i, half, p, d), a1 = plane_alpha(i + 1, half, p, d);
    lo = a0 < a1 ? a0 : a1;
    hi = a0 < a1 ? a1 : a0;
    return true;
  }
  int c = (int)floor(dadd(p, half));
  c = c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
  lo = -INFINITY;
  hi = INFINITY;
  return c == i;
}

__global__ void matfree_backproject_kernel(GeomDev g, const double4* rs, const float* y, float* x,
                                           int S, int64_t nray) {
  const int n = g.n;
  const int64_t npix = (int64_t)n * n;
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int ix = (int)(pix % n), iy = (int)(pix / n);
  const double half = dmul(0.5, (double)n);
  // pixel centre, for the window of candidate bins only
  const double xc = (double)ix - half + 0.5, yc = (double)iy - half + 0.5;
  const double c0 = 0.5 * (double)(g.nd - 1);
  for (int s0 = 0; s0 < S; s0 += kMfSlices) {
    const int ns = min(kMfSlices, S - s0);
    float acc[kMfSlices];
#pragma unroll
    for (int q = 0; q < kMfSlices; ++q) acc[q] = 0.0f;
    for (int k = 0; k < g.m; ++k) {
      const double c = g.cs[2 * k], sn = g.cs[2 * k + 1];
      const double dx = -sn, dy = c;
      // bins whose line can meet the pixel: |t_j - t_c| <= (|c| + |s|) / 2,
      // one more bin on each side (the plane test below decides)
      const double tc = xc * c + yc * sn, w = 0.5 * (fabs(c) + fabs(sn));
      double jlo = (tc - w - g.doff) / g.dspace + c0, jhi = (tc + w - g.doff) / g.dspace + c0;
      if (jlo > jhi) {
        const double t = jlo;
        jlo = jhi;
        jhi = t;
      }
      const int j0 = max(0, (int)floor(jlo) - 1), j1 = min(g.nd - 1, (int)ceil(jhi) + 1);
      for (int j = j0; j <= j1; ++j) {
        const int64_t ray = (int64_t)k * g.nd + j;
        const double4 q = rs[ray];   // px, py, amin, amax
        if (!(q.z <= q.w)) continue;
        double xlo, xhi, ylo, yhi;
        if (!pixel_axis(ix, n, half, q.x, dx, xlo, xhi)) continue;
        if (!pixel_axis(iy, n, half, q.y, dy, ylo, yhi)) continue;
        double a = xlo > ylo ? xlo : ylo, b = xhi < yhi ? xhi : yhi;
        a = a > q.z ? a : q.z;
        b = b < q.w ? b : q.w;
        const double len = dsub(b, a);
        if (!(len >= g.min_seg)) continue;
        const double mid = dmul(dadd(a, b), 0.5);
        int px = (int)floor(dadd(dadd(q.x, dmul(mid, dx)), half));
        int py = (int)floor(dadd(dadd(q.y, dmul(mid, dy)), half));
        px = px < 0 ? 0 : (px > n - 1 ? n - 1 : px);
        py = py < 0 ? 0 : (py > n - 1 ? n - 1 : py);
        if (px != ix || py != iy) continue;
        const float l = (float)len;
#pragma unroll
        for (int q2 = 0; q2 < kMfSlices; ++q2)
          if (q2 < ns) acc[q2] = fmaf(l, __ldg(y + (size_t)(s0 + q2) * nray + ray), acc[q2]);
      }
    }
    for (int q = 0; q < ns; ++q) x[(size_t)(s0 + q) * npix + pix] = acc[q];
  }
}

xct_status matfree_backproject(const Plan& p, const double* cs_dev, const float* y, float* x, int S,
                               cudaStream_t s) {
  const xct_geometry& g = p.g;
  GeomDev gd{g.n, g.n_angles, g.n_det, g.det_spacing, g.det_offset, g.min_seg, cs_dev};
  Arena tmp(s);
  double4* rs;
  XCT_TRY(tmp.get(&rs, p.nray));
  matfree_ray_setup_kernel<<<grid_for(p.nray, 256), 256, 0, s>>>(gd, p.nray, rs);
  matfree_backproject_kernel<<<grid_for(p.npix, 128), 128, 0, s>>>(gd, rs, y, x, S, p.nray);
  count_launch(2);
  XCT_TRY_CUDA(cudaGetLastError());
  XCT_TRY_CUDA(cudaStreamSynchronize(s));   // rs is released next
  return XCT_OK;
}

xct_status matfree_project(const Plan& p, const double* cs_dev, const float* x, float* y, int S,
                           cudaStream_t s) {
  const xct_geometry& g = p.g;
  GeomDev gd{g.n, g.n_angles, g.n_det, g.det_spacing, g.det_offset, g.min_seg, cs_dev};
  matfree_project_kernel<<<grid_for(p.nray, 128), 128, 0, s>>>(gd, x, y, S, p.nray);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status build_plan(Plan& p, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  const xct_geometry& g = p.g;
  p.npix = (int64_t)g.n * g.n;
  p.nray = (int64_t)g.n_angles * g.n_det;
  p.mat_scale_exp = half_values(p.storage) ? 15 : 0;
  const int T = g.hilbert_tile > 0 ? g.hilbert_tile : 8;
  Arena& keep = p.mem;
  keep.stream = s;
  Arena tmp(s);

  double* cs_dev;
  XCT_TRY(tmp.get(&cs_dev, 2 * (size_t)g.n_angles));
  XCT_TRY_CUDA(cudaMemcpyAsync(cs_dev, p.cs.data(), sizeof(double) * 2 * g.n_angles,
                               cudaMemcpyHostToDevice, s));
  XCT_TRY(keep.get(&p.err, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), s));
  XCT_TRY(keep.get(&p.pix_order, p.npix));
  XCT_TRY(keep.get(&p.pix_inv, p.npix));
  XCT_TRY(keep.get(&p.ray_order, p.nray));
  XCT_TRY(keep.get(&p.ray_inv, p.nray));
  // Inside a tile: pixels in 2 x 2 groups, rays angle-fastest.  Four
  // consecutive rows of A (or A^T) form one quad of the packed layout, padded
  // to its longest row per stage; neighbouring angles through one bin (and
  // 2 x 2 pixel groups) cross a stage's pixels (rays) more evenly than four
  // neighbouring bins (a 1 x 4 pixel run), so less padding.
  XCT_TRY(make_order(g.n, g.n, T, kInnerQuad, p.pix_order, p.pix_inv, s));
  XCT_TRY(make_order(g.n_det, g.n_angles, T, kInnerCol, p.ray_order, p.ray_inv, s));

  GeomDev gd{g.n, g.n_angles, g.n_det, g.det_spacing, g.det_offset, g.min_seg, cs_dev};
  int32_t* cnt;
  int64_t* rowptr;
  XCT_TRY(tmp.get(&cnt, p.nray));
  Arena f64(s);  // FP64 CSR / CSC, kept only with XCT_PLAN_KEEP_F64
  XCT_TRY(f64.get(&rowptr, p.nray + 1));
  siddon_count_kernel<<<grid_for(p.nray, 128), 128, 0, s>>>(gd, p.ray_inv, p.nray, cnt);
  count_launch();
  XCT_TRY(exclusive_scan_i32(cnt, rowptr, p.nray, s));
  XCT_TRY_CUDA(cudaMemcpyAsync(&p.nnz, rowptr + p.nray, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  int32_t* col;
  double* val;
  XCT_TRY(f64.get(&col, p.nnz));
  XCT_TRY(f64.get(&val, p.nnz));
  siddon_fill_kernel<<<grid_for(p.nray, 128), 128, 0, s>>>(gd, p.ray_inv, p.pix_order, p.nray,
                                                          rowptr, col, val);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());

  int64_t* colptr;
  int32_t* trow;
  double* tval;
  XCT_TRY(f64.get(&colptr, p.npix + 1));
  XCT_TRY(f64.get(&trow, p.nnz));
  XCT_TRY(f64.get(&tval, p.nnz));
  XCT_TRY(transpose(rowptr, col, val, p.nray, p.npix, p.nnz, colptr, trow, tval, s));

  // Stage capacity of each matrix: the pipeline buffers (128-byte staged
  // rows plus the stage's packed entries) must fit in shared memory; a layout
  // whose largest stage does not fit is rebuilt with a smaller capacity.
  // With XCT_PLAN_AUTOTUNE the capacity is also chosen by timing the
  // product on the widest slice tile among a few candidates.
  CsrView ma{rowptr, col, val, p.nray, p.npix};
  CsrView mt{colptr, trow, tval, p.npix, p.nray};
  const int32_t cap0 = p.storage == XCT_F32 ? kPipeCap32 : kPipeCap16;
  auto fitted = [&](const CsrView& m, int32_t cap, Layout& L, Arena& mem) -> xct_status {
    for (int attempt = 0;; ++attempt) {
      Arena lm(s);
      Layout t;
      XCT_TRY(build_layout(m, p.nnz, p.storage, cap, t, lm, s, -1, kEntryRowBytes,
                           (p.flags & XCT_PLAN_NARROW_TILES) != 0));
      if (kPipeBufs * pipe_buffer_bytes(t, 128) <= kPipeSmemLimit || attempt == 3 || cap <= 64) {
        L = t;
        lm.move_to(mem);
        return XCT_OK;
      }
      cap = (cap * 3 / 4) & ~3;   // multiple of 4: stage lists stay 16-byte aligned
    }
  };
  for (int which = 0; which < 2; ++which) {
    const CsrView& m = which == 0 ? ma : mt;
    Layout& out = which == 0 ? p.la : p.lat;
    if (!(p.flags & XCT_PLAN_AUTOTUNE)) {
      Arena mem(s);
      XCT_TRY(fitted(m, cap0, out, mem));
      mem.move_to(keep);
      continue;
    }
    double best_ms = 1e300;
    Arena best_mem(s);
    for (int32_t cand : {cap0, (cap0 * 4 / 5) & ~3, (cap0 * 3 / 5) & ~3}) {
      Arena mem(s);
      Layout L;
      XCT_TRY(fitted(m, cand, L, mem));
      double ms = 0.0;
      XCT_TRY(time_product(L, p, s, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        best_mem.release();
        mem.move_to(best_mem);
        out = L;
      }
    }
    best_mem.move_to(keep);
  }
  const int32_t cap_used = p.la.cap;
  // wide-stage layouts for products of few slices (16-byte staged rows):
  // stages of up to kWideCapA / kWideCapAT rows, gaps of up to kWideGap unreferenced rows
  // filled, offsets at 16 bytes per row; the entries stay in global memory
  if (p.flags & XCT_PLAN_FEW_SLICES) {
    for (int which = 0; which < 2; ++which) {
      Arena mem(s);
      Layout& out = which == 0 ? p.law : p.latw;
      XCT_TRY(build_layout(which == 0 ? ma : mt, p.nnz, p.storage, which == 0 ? kWideCapA : kWideCapAT, out, mem, s, kWideGap,
                           kWideRowBytes));
      mem.move_to(keep);
    }
    p.la.wide = &p.law;
    p.lat.wide = &p.latw;
  }
  // paired layouts for 64-slice tiles of 16-bit slices, kept where their
  // stage buffers fit the persistent product (else those tiles use the plain
  // layouts)
  if (p.flags & XCT_PLAN_PAIRED_ROWS) {
    int dummy_work = 0, dummy_err = 0;
    for (int which = 0; which < 2; ++which) {
      Layout& base = which == 0 ? p.la : p.lat;
      Layout& out = which == 0 ? p.lap : p.latp;
      Arena mem(s);
      XCT_TRY(build_paired_layout(base, out, mem, s));
      SpmmArgs probe{};
      probe.L = &out;
      probe.st = kEntryRowBytes / 2;
      probe.ntiles = 1;
      probe.storage = p.storage;
      probe.work = &dummy_work;   // only tested for null
      probe.err = &dummy_err;
      if (spmm_pipe_applies(probe)) {
        mem.move_to(keep);
        base.paired = &out;
      } else {
        mem.release();
        out = Layout{};
      }
    }
  }

  if (p.flags & XCT_PLAN_KEEP_F64) {
    p.a_rowptr = rowptr; p.a_col = col; p.a_val = val;
    p.t_rowptr = colptr; p.t_col = trow; p.t_val = tval;
    f64.move_to(keep);
  }
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  tmp.release();
  f64.release();
  XCT_TRY_CUDA(cudaStreamSynchronize(s));

  auto t1 = std::chrono::steady_clock::now();
  xct_stats& st = p.stats;
  st.n_rays = p.nray;
  st.n_pix = p.npix;
  st.nnz = p.nnz;
  st.storage = p.storage;
  st.rows_per_block = kRowsPerBlock;
  st.stage_capacity = cap_used;
  st.stage_capacity_at = p.lat.cap;
  st.stages_a = p.la.nstages;
  st.stages_at = p.lat.nstages;
  st.slots_a = p.la.nslots;
  st.slots_at = p.lat.nslots;
  st.bytes_a = p.la.bytes;
  st.bytes_at = p.lat.bytes;
  st.slots_a_paired = p.la.paired ? p.la.paired->nslots : 0;
  st.slots_at_paired = p.lat.paired ? p.lat.paired->nslots : 0;
  st.gathers_a_paired = p.la.paired ? p.la.paired->gathers : 0;
  st.gathers_at_paired = p.lat.paired ? p.lat.paired->gathers : 0;
  st.plan_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  return XCT_OK;
}

// ---------------------------------------------------------------------------
// export (verification): canonical natural-order CSR on the host
// ---------------------------------------------------------------------------

namespace {

struct Coo { int32_t r, c; double v; };

xct_status to_canonical(std::vector<Coo>& coo, int64_t nrows, int64_t* rowptr, int32_t* col,
                        double* val, int64_t* nnz) {
  std::sort(coo.begin(), coo.end(), [](const Coo& a, const Coo& b) {
    return a.r != b.r ? a.r < b.r : a.c < b.c;
  });
  *nnz = (int64_t)coo.size();
  if (!rowptr) return XCT_OK;
  for (int64_t r = 0; r <= nrows; ++r) rowptr[r] = 0;
  for (size_t i = 0; i < coo.size(); ++i) {
    rowptr[coo[i].r + 1]++;
    col[i] = coo[i].c;
    val[i] = coo[i].v;
  }
  for (int64_t r = 0; r < nrows; ++r) rowptr[r + 1] += rowptr[r];
  return XCT_OK;
}

template <class T>
xct_status d2h(std::vector<T>& h, const T* d, int64_t n) {
  h.resize((size_t)std::max<int64_t>(n, 0));
  if (n > 0) XCT_TRY_CUDA(cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost));
  return XCT_OK;
}

double stored_value(const Plan& p, uint16_t h) {
  if (half_values(p.storage)) {
    __half_raw hr;
    hr.x = h;
    return (double)__half2float(__half(hr)) * ldexp(1.0, -p.mat_scale_exp);
  }
  const uint32_t f = (uint32_t)h << 16;
  float ff;
  memcpy(&ff, &f, 4);
  return (double)ff * ldexp(1.0, -p.mat_scale_exp);
}

// The entries of a paired layout (placement described with kPairUA): every
// half of a slot whose offset is not the zero slot's is an entry; a shared
// slot gives one entry to each row of its pair at the same column.
xct_status decode_paired(const Layout& L, const Plan& p, int64_t nrows, const std::vector<int32_t>& row_inv,
                         const std::vector<int32_t>& col_inv, std::vector<Coo>& coo) {
  std::vector<int64_t> bs, sp;
  std::vector<int32_t> px;
  std::vector<Seg> sg;
  std::vector<unsigned long long> e8;
  XCT_TRY(d2h(bs, L.blk_stage, (int64_t)L.nblocks + 1));
  XCT_TRY(d2h(sp, L.stage_pix, L.nstages + 1));
  XCT_TRY(d2h(px, L.pix, L.footprint));
  XCT_TRY(d2h(sg, L.seg, L.nstages * kQuads));
  XCT_TRY(d2h(e8, static_cast<const unsigned long long*>(L.ent), L.nslots));
  const uint32_t zero = (uint32_t)L.cap * kEntryRowBytes;
  for (int32_t b = 0; b < L.nblocks; ++b)
    for (int64_t st = bs[b]; st < bs[b + 1]; ++st)
      for (int q = 0; q < kQuads; ++q) {
        const Seg& s = sg[st * kQuads + q];
        const int ga = (std::max(s.cnt[0], s.cnt[2]) + kPairUA - 1) / kPairUA;
        for (int pr = 0; pr < 2; ++pr)
          for (int region = 0; region < 2; ++region) {
            const int per = region == 0 ? kPairUA : kPairUB;
            const int64_t r0 = s.off + (region == 0 ? 0 : (int64_t)ga * 4 * kPairUA);
            for (int c = 0; c < s.cnt[2 * pr + region]; ++c)
              for (int e = 0; e < 2; ++e) {
                const int64_t slot = r0 + (int64_t)(c / per) * 4 * per + (2 * pr + e) * per + c % per;
                if (slot < 0 || slot >= L.nslots) {
                  set_error("paired layout: slot outside the entries (block %d stage %lld)", b, (long long)st);
                  return XCT_ERR_CUDA;
                }
                const uint32_t half[2] = {(uint32_t)(e8[slot] & 0xffffffffu), (uint32_t)(e8[slot] >> 32)};
                for (int h = 0; h < 2; ++h) {
                  uint32_t off = half[h] >> 16;
                  if (region == 0) off = half[0] >> 16;   // a shared slot's column is its first half's
                  if (off == zero) continue;
                  const uint32_t idx = off / (uint32_t)kEntryRowBytes;
                  const int64_t row = (int64_t)b * kRowsPerBlock + q * 4 + 2 * pr + h;
                  if (off % (uint32_t)kEntryRowBytes || idx >= (uint32_t)(sp[st + 1] - sp[st]) || row >= nrows) {
                    set_error("paired layout holds an out-of-range entry (block %d stage %lld)", b, (long long)st);
                    return XCT_ERR_CUDA;
                  }
                  coo.push_back({row_inv[row], col_inv[px[sp[st] + idx]],
                                 stored_value(p, (uint16_t)(half[h] & 0xffffu))});
                }
              }
          }
      }
  return XCT_OK;
}

}  // namespace

xct_status export_matrix(Plan& p, int what, int64_t* rowptr, int32_t* col, double* val,
                         int64_t* nnz) {
  const bool tr = (what == XCT_EXPORT_AT_F64 || what == XCT_EXPORT_AT_STORED || what == XCT_EXPORT_AT_PAIRED);
  const int64_t nrows = tr ? p.npix : p.nray;
  std::vector<int32_t> row_inv, col_inv;  // ordered id -> natural id
  XCT_TRY(d2h(row_inv, tr ? p.pix_inv : p.ray_inv, nrows));
  XCT_TRY(d2h(col_inv, tr ? p.ray_inv : p.pix_inv, tr ? p.nray : p.npix));
  std::vector<Coo> coo;
  if (what == XCT_EXPORT_A_F64 || what == XCT_EXPORT_AT_F64) {
    if (!(p.flags & XCT_PLAN_KEEP_F64)) {
      set_error("FP64 export needs a plan built with XCT_PLAN_KEEP_F64");
      return XCT_ERR_INVALID;
    }
    std::vector<int64_t> rp;
    std::vector<int32_t> cc;
    std::vector<double> vv;
    XCT_TRY(d2h(rp, tr ? p.t_rowptr : p.a_rowptr, nrows + 1));
    XCT_TRY(d2h(cc, tr ? p.t_col : p.a_col, p.nnz));
    XCT_TRY(d2h(vv, tr ? p.t_val : p.a_val, p.nnz));
    coo.reserve((size_t)p.nnz);
    for (int64_t r = 0; r < nrows; ++r)
      for (int64_t e = rp[r]; e < rp[r + 1]; ++e) coo.push_back({row_inv[r], col_inv[cc[e]], vv[e]});
  } else if (what == XCT_EXPORT_A_PAIRED || what == XCT_EXPORT_AT_PAIRED) {
    const Layout* LP = (tr ? p.lat : p.la).paired;
    if (!LP) {
      set_error("paired export needs a plan built with XCT_PLAN_PAIRED_ROWS whose paired layouts fit");
      return XCT_ERR_INVALID;
    }
    XCT_TRY(decode_paired(*LP, p, nrows, row_inv, col_inv, coo));
  } else {
    const Layout& L = tr ? p.lat : p.la;
    std::vector<int64_t> bs, sp;
    std::vector<int32_t> px;
    std::vector<Seg> sg;
    XCT_TRY(d2h(bs, L.blk_stage, (int64_t)L.nblocks + 1));
    XCT_TRY(d2h(sp, L.stage_pix, L.nstages + 1));
    XCT_TRY(d2h(px, L.pix, L.footprint));
    XCT_TRY(d2h(sg, L.seg, L.nstages * kQuads));
    std::vector<uint32_t> e4;
    std::vector<unsigned long long> e8;
    if (L.ebytes == 4) XCT_TRY(d2h(e4, static_cast<const uint32_t*>(L.ent), L.nslots));
    else XCT_TRY(d2h(e8, static_cast<const unsigned long long*>(L.ent), L.nslots));
    const double unscale = ldexp(1.0, -p.mat_scale_exp);
    for (int32_t b = 0; b < L.nblocks; ++b) {
      for (int64_t st = bs[b]; st < bs[b + 1]; ++st) {
        for (int q = 0; q < kQuads; ++q) {
          const Seg& s = sg[st * kQuads + q];
          for (int g = 0; g < 4; ++g) {
            int64_t row = (int64_t)b * kRowsPerBlock + q * 4 + g;
            for (int k = 0; k < s.cnt[g]; ++k) {
              int64_t slot = s.off + (k >> 2) * 16 + g * 4 + (k & 3);
              uint32_t idx;
              double v;
              uint32_t off;
              if (L.ebytes == 4) {
                uint32_t w = e4[slot];
                off = w >> 16;
                uint16_t h = (uint16_t)(w & 0xffffu);
                if (half_values(p.storage)) {
                  __half_raw hr;
                  hr.x = h;
                  v = (double)__half2float(__half(hr));
                } else {
                  uint32_t f = (uint32_t)h << 16;
                  float ff;
                  memcpy(&ff, &f, 4);
                  v = ff;
                }
              } else {
                unsigned long long w = e8[slot];
                off = (uint32_t)(w & 0xffffffffu);
                uint32_t f = (uint32_t)(w >> 32);
                float ff;
                memcpy(&ff, &f, 4);
                v = ff;
              }
              idx = off / (uint32_t)L.unit;
              if (off % (uint32_t)L.unit || idx >= (uint32_t)(sp[st + 1] - sp[st]) || row >= nrows) {
                set_error("packed layout holds an out-of-range entry (block %d stage %lld)", b,
                          (long long)st);
                return XCT_ERR_CUDA;
              }
              int32_t c = px[sp[st] + idx];
              coo.push_back({row_inv[row], col_inv[c], v * unscale});
            }
          }
        }
      }
    }
  }
  return to_canonical(coo, nrows, rowptr, col, val, nnz);
}

}  // namespace xct

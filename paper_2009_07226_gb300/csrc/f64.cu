// Double-precision comparison path.  Sec. V compares the reconstruction in
// double, single, half and mixed precision (speed and convergence); this is
// the double form: FP64 matrix values (the plan's kept FP64 CSR of A and of
// its explicit transpose, ordered ids), FP64 vectors, FP64 FMAs, and the
// CGLS of Sec. II-C with FP64 scalars.  GB300 runs FP64 FMAs at a small
// fraction of its FP32 rate, so these products are bound by that rate; the
// path is a yardstick for the single-precision and 16-bit forms, not a fast
// path.
//
// Internal vector layout: [rows (ordered ids)][S] float64, the slices of one
// row contiguous (one warp reads a row's slices as one coalesced segment).
#include <math.h>

#include <vector>

#include "xct_internal.cuh"

namespace xct {
namespace {

constexpr int kF64Threads = 256;                 // 8 warps
constexpr int kF64Warps = kF64Threads / 32;
constexpr int kF64Chunk = 64;                    // slices per product pass (2 per lane)
constexpr int kF64Blocks = 152 * 8;              // fixed grid: deterministic partial sums

int f64_grid(int64_t rows) {
  const int64_t want = (rows + kF64Warps - 1) / kF64Warps;
  return (int)(want < kF64Blocks ? (want > 0 ? want : 1) : kF64Blocks);
}

// in[i][s] = nat[s][inv[i]]: natural slice-major -> internal
__global__ void f64_gather_kernel(const double* __restrict__ nat, double* __restrict__ in,
                                  const int32_t* __restrict__ inv, int64_t rows, int S) {
  const int64_t n = rows * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / S;
    const int s = (int)(t - i * S);
    in[t] = nat[(size_t)s * rows + inv[i]];
  }
}

// nat[s][inv[i]] = in[i][s]
__global__ void f64_scatter_kernel(const double* __restrict__ in, double* __restrict__ nat,
                                   const int32_t* __restrict__ inv, int64_t rows, int S) {
  const int64_t n = rows * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / S;
    const int s = (int)(t - i * S);
    nat[(size_t)s * rows + inv[i]] = in[t];
  }
}

// One pass of Y = A X over slices [s0, s0 + sc), sc <= 64: one warp per row
// (grid-stride), lane l accumulating slices s0 + l and s0 + l + 32.  The
// row's entries are read 32 at a time (coalesced) and broadcast by shuffles.
// dot (nullable): per-block sums of y^2 per slice, [S][gridDim.x].
__global__ void __launch_bounds__(kF64Threads)
    f64_spmm_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                    const double* __restrict__ val, int64_t nrows, const double* __restrict__ x,
                    double* __restrict__ y, int S, int s0, int sc, double* dot) {
  __shared__ double red[kF64Warps][kF64Chunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool on0 = lane < sc, on1 = lane + 32 < sc;
  double sq0 = 0.0, sq1 = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * kF64Warps + warp; r < nrows;
       r += (int64_t)gridDim.x * kF64Warps) {
    double a0 = 0.0, a1 = 0.0;
    const int64_t b = rowptr[r], e = rowptr[r + 1];
    for (int64_t j0 = b; j0 < e; j0 += 32) {
      const int64_t j = j0 + lane;
      const int c = j < e ? col[j] : 0;
      const double v = j < e ? val[j] : 0.0;
      const int n = (int)(e - j0 < 32 ? e - j0 : 32);
      for (int t = 0; t < n; ++t) {
        const int ct = __shfl_sync(0xffffffffu, c, t);
        const double vt = __shfl_sync(0xffffffffu, v, t);
        const double* xr = x + (size_t)ct * S + s0;
        if (on0) a0 = fma(vt, xr[lane], a0);
        if (on1) a1 = fma(vt, xr[lane + 32], a1);
      }
    }
    double* yr = y + (size_t)r * S + s0;
    if (on0) {
      yr[lane] = a0;
      sq0 = fma(a0, a0, sq0);
    }
    if (on1) {
      yr[lane + 32] = a1;
      sq1 = fma(a1, a1, sq1);
    }
  }
  if (dot) {
    red[warp][lane] = sq0;
    red[warp][lane + 32] = sq1;
    __syncthreads();
    for (int s = threadIdx.x; s < sc; s += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < kF64Warps; ++w) t += red[w][s];
      dot[(size_t)(s0 + s) * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Per-block sums of v^2 per slice over slices [s0, s0 + sc) of v [rows][S],
// written to part [S][gridDim.x] (the same row-to-block map as the product).
__global__ void __launch_bounds__(kF64Threads)
    f64_sqnorm_kernel(const double* __restrict__ v, int64_t rows, int S, int s0, int sc,
                      double* part) {
  __shared__ double red[kF64Warps][kF64Chunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool on0 = lane < sc, on1 = lane + 32 < sc;
  double sq0 = 0.0, sq1 = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * kF64Warps + warp; r < rows;
       r += (int64_t)gridDim.x * kF64Warps) {
    const double* vr = v + (size_t)r * S + s0;
    if (on0) sq0 = fma(vr[lane], vr[lane], sq0);
    if (on1) sq1 = fma(vr[lane + 32], vr[lane + 32], sq1);
  }
  red[warp][lane] = sq0;
  red[warp][lane + 32] = sq1;
  __syncthreads();
  for (int s = threadIdx.x; s < sc; s += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kF64Warps; ++w) t += red[w][s];
    part[(size_t)(s0 + s) * gridDim.x + blockIdx.x] = t;
  }
}

// v[i][s] += sign * coef[s] * w[i][s]
__global__ void f64_axpy_kernel(double* __restrict__ v, const double* __restrict__ w,
                                const double* __restrict__ coef, double sign, int64_t rows,
                                int S) {
  const int64_t n = rows * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % S);
    v[t] = fma(sign * coef[s], w[t], v[t]);
  }
}

// p[i][s] = sv[i][s] + beta[s] * p[i][s]
__global__ void f64_xpby_kernel(double* __restrict__ p, const double* __restrict__ sv,
                                const double* __restrict__ beta, int64_t rows, int S) {
  const int64_t n = rows * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % S);
    p[t] = fma(beta[s], p[t], sv[t]);
  }
}

// v = a - b
__global__ void f64_sub_kernel(double* __restrict__ v, const double* __restrict__ b,
                               int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    v[t] -= b[t];
}

struct F64Scalars {
  double *gamma, *alpha, *beta;
  int *active, *active0;
};

__device__ double sum_fixed(const double* p, int nb) {
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += p[b];
  return t;
}

// one thread per slice.  mode 0: start (gamma = ||s||^2, log[0]); mode 1:
// alpha = gamma / ||q||^2; mode 2: beta = gamma' / gamma, log[k].  A slice
// whose gamma or delta is exactly 0 stops (alpha = beta = 0 from then on).
__global__ void f64_scalars_kernel(int mode, const double* part, int nb, const double* rpart,
                                   int nbr, F64Scalars sc, int S, double* log_k) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double g = sum_fixed(part + (size_t)s * nb, nb);
  if (mode == 0) {
    const int act = g > 0.0;
    sc.gamma[s] = g;
    sc.active[s] = act;
    sc.active0[s] = act;
    sc.beta[s] = 0.0;
  } else if (mode == 1) {
    const int act = sc.active[s] && g > 0.0;
    sc.active[s] = act;
    sc.alpha[s] = act ? sc.gamma[s] / g : 0.0;
    return;
  } else {
    const int act = sc.active[s];
    sc.beta[s] = act ? g / sc.gamma[s] : 0.0;
    if (act) sc.gamma[s] = g;
    sc.active[s] = act && g > 0.0;
  }
  if (log_k) {
    const double rr = sum_fixed(rpart + (size_t)s * nbr, nbr);
    log_k[(size_t)s * 2] = sqrt(rr);
    log_k[(size_t)s * 2 + 1] = sqrt(g);
  }
}

int vec_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

struct Csr64 {
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  int64_t nrows;
};

// Y = A X on the internal layout; dot (nullable) as f64_spmm_kernel
xct_status spmm64(const Csr64& m, const double* x, double* y, int S, double* dot, cudaStream_t s) {
  const int grid = f64_grid(m.nrows);
  for (int s0 = 0; s0 < S; s0 += kF64Chunk) {
    const int sc = S - s0 < kF64Chunk ? S - s0 : kF64Chunk;
    f64_spmm_kernel<<<grid, kF64Threads, 0, s>>>(m.rowptr, m.col, m.val, m.nrows, x, y, S, s0, sc,
                                                 dot);
    count_launch();
  }
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status sqnorm64(const double* v, int64_t rows, int S, double* part, cudaStream_t s) {
  const int grid = f64_grid(rows);
  for (int s0 = 0; s0 < S; s0 += kF64Chunk) {
    const int sc = S - s0 < kF64Chunk ? S - s0 : kF64Chunk;
    f64_sqnorm_kernel<<<grid, kF64Threads, 0, s>>>(v, rows, S, s0, sc, part);
    count_launch();
  }
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status gather64(const double* nat, double* in, const int32_t* inv, int64_t rows, int S,
                    cudaStream_t s) {
  f64_gather_kernel<<<vec_grid(rows * S), 256, 0, s>>>(nat, in, inv, rows, S);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status scatter64(const double* in, double* nat, const int32_t* inv, int64_t rows, int S,
                     cudaStream_t s) {
  f64_scatter_kernel<<<vec_grid(rows * S), 256, 0, s>>>(in, nat, inv, rows, S);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status have_f64(const Plan& p) {
  if (!p.a_val || !p.t_val) {
    set_error("the FP64 path needs a plan built with XCT_PLAN_KEEP_F64");
    return XCT_ERR_INVALID;
  }
  return XCT_OK;
}

}  // namespace

xct_status f64_apply(Plan& p, bool transposed, const double* in, double* out, int S,
                     cudaStream_t s) {
  XCT_TRY(have_f64(p));
  XCT_TRY_CUDA(cudaSetDevice(p.device));
  const Csr64 m = transposed ? Csr64{p.t_rowptr, p.t_col, p.t_val, p.npix}
                             : Csr64{p.a_rowptr, p.a_col, p.a_val, p.nray};
  const int64_t nin = transposed ? p.nray : p.npix, nout = m.nrows;
  Arena ar(s);
  double *X, *Y;
  XCT_TRY(ar.get(&X, (size_t)nin * S));
  XCT_TRY(ar.get(&Y, (size_t)nout * S));
  XCT_TRY(gather64(in, X, transposed ? p.ray_inv : p.pix_inv, nin, S, s));
  XCT_TRY(spmm64(m, X, Y, S, nullptr, s));
  XCT_TRY(scatter64(Y, out, transposed ? p.pix_inv : p.ray_inv, nout, S, s));
  return XCT_OK;
}

xct_status f64_cgls(Plan& p, const double* y, double* x, int S, int iters, bool x0,
                    double* log, int* any_active, cudaStream_t s) {
  XCT_TRY(have_f64(p));
  XCT_TRY_CUDA(cudaSetDevice(p.device));
  const Csr64 A{p.a_rowptr, p.a_col, p.a_val, p.nray};
  const Csr64 AT{p.t_rowptr, p.t_col, p.t_val, p.npix};
  const int64_t npix = p.npix, nray = p.nray;
  const int nbA = f64_grid(nray), nbT = f64_grid(npix);
  Arena ar(s);
  double *X, *R, *P, *Q, *Sv, *dpart, *gpart, *rpart;
  F64Scalars sc{};
  XCT_TRY(ar.get(&X, (size_t)npix * S));
  XCT_TRY(ar.get(&P, (size_t)npix * S));
  XCT_TRY(ar.get(&Sv, (size_t)npix * S));
  XCT_TRY(ar.get(&R, (size_t)nray * S));
  XCT_TRY(ar.get(&Q, (size_t)nray * S));
  XCT_TRY(ar.get(&dpart, (size_t)S * nbA));
  XCT_TRY(ar.get(&rpart, (size_t)S * nbA));
  XCT_TRY(ar.get(&gpart, (size_t)S * nbT));
  XCT_TRY(ar.get(&sc.gamma, S));
  XCT_TRY(ar.get(&sc.alpha, S));
  XCT_TRY(ar.get(&sc.beta, S));
  XCT_TRY(ar.get(&sc.active, S));
  XCT_TRY(ar.get(&sc.active0, S));
  const int sg = (S + 127) / 128;

  // r = y - A x0 (or y);  s = A^T r;  p = s;  gamma = ||s||^2
  XCT_TRY(gather64(y, R, p.ray_inv, nray, S, s));
  if (x0) {
    XCT_TRY(gather64(x, X, p.pix_inv, npix, S, s));
    XCT_TRY(spmm64(A, X, Q, S, nullptr, s));
    f64_sub_kernel<<<vec_grid(nray * S), 256, 0, s>>>(R, Q, nray * S);
    count_launch();
  } else {
    XCT_TRY_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * npix * S, s));
  }
  XCT_TRY(sqnorm64(R, nray, S, rpart, s));
  XCT_TRY(spmm64(AT, R, Sv, S, gpart, s));
  f64_scalars_kernel<<<sg, 128, 0, s>>>(0, gpart, nbT, rpart, nbA, sc, S, log);
  count_launch();
  XCT_TRY_CUDA(cudaMemcpyAsync(P, Sv, sizeof(double) * npix * S, cudaMemcpyDeviceToDevice, s));
  for (int k = 1; k <= iters; ++k) {
    // q = A p;  alpha = gamma / ||q||^2;  x += alpha p;  r -= alpha q
    XCT_TRY(spmm64(A, P, Q, S, dpart, s));
    f64_scalars_kernel<<<sg, 128, 0, s>>>(1, dpart, nbA, nullptr, 0, sc, S, nullptr);
    count_launch();
    f64_axpy_kernel<<<vec_grid(npix * S), 256, 0, s>>>(X, P, sc.alpha, 1.0, npix, S);
    f64_axpy_kernel<<<vec_grid(nray * S), 256, 0, s>>>(R, Q, sc.alpha, -1.0, nray, S);
    count_launch(2);
    XCT_TRY(sqnorm64(R, nray, S, rpart, s));
    // s = A^T r;  beta = gamma' / gamma;  p = s + beta p
    XCT_TRY(spmm64(AT, R, Sv, S, gpart, s));
    f64_scalars_kernel<<<sg, 128, 0, s>>>(2, gpart, nbT, rpart, nbA, sc, S,
                                          log ? log + (size_t)k * S * 2 : nullptr);
    count_launch();
    f64_xpby_kernel<<<vec_grid(npix * S), 256, 0, s>>>(P, Sv, sc.beta, npix, S);
    count_launch();
  }
  XCT_TRY_CUDA(cudaGetLastError());
  XCT_TRY(scatter64(X, x, p.pix_inv, npix, S, s));
  std::vector<int> act((size_t)S);
  XCT_TRY_CUDA(cudaMemcpyAsync(act.data(), sc.active0, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  int any = 0;
  for (int i = 0; i < S; ++i) any |= act[i];
  *any_active = any;
  return XCT_OK;
}

}  // namespace xct

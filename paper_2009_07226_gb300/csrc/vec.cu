// Vector kernels around the products: layout conversion between the caller's
// slice-major natural order and the internal [tile][ordered row][slice]
// layout, and the CGLS vector updates and FP64 scalars (Eq. 1 with R = 0,
// CGLS form with one initial back projection, per-slice scalars).
#include "ff.cuh"
#include "xct_internal.cuh"
#include "xct_vec.cuh"

namespace xct {
namespace {

constexpr int kConvRows = 32;     // ordered rows per conversion block
constexpr int kConvThreads = 256;

// natural [S][rows] -> internal [ntiles][rows][st]; slices >= S are zero.
// Optionally accumulates max |v| per slice into max_bits (float bits).
__global__ void __launch_bounds__(kConvThreads) to_internal_kernel(
    const float* __restrict__ nat, float* __restrict__ out, const int32_t* __restrict__ inv,
    int64_t rows, int S, int st, uint32_t* __restrict__ max_bits) {
  extern __shared__ float tile_buf[];  // [kConvRows][st + 1]
  __shared__ uint32_t smax[64];
  const int64_t h0 = (int64_t)blockIdx.x * kConvRows;
  const int t = blockIdx.y;
  const int nr = (int)min((int64_t)kConvRows, rows - h0);
  for (int i = threadIdx.x; i < st; i += blockDim.x) smax[i] = 0;
  __syncthreads();
  // read: h fastest so the natural ids of a Hilbert tile row are contiguous
  for (int i = threadIdx.x; i < kConvRows * st; i += blockDim.x) {
    const int sl = i / kConvRows, r = i % kConvRows;
    const int s = t * st + sl;
    float v = 0.0f;
    if (r < nr && s < S) v = nat[(size_t)s * rows + inv[h0 + r]];
    tile_buf[r * (st + 1) + sl] = v;
    if (max_bits) atomicMax(&smax[sl], __float_as_uint(fabsf(v)));
  }
  __syncthreads();
  float* dst = out + ((size_t)t * rows + h0) * st;
  for (int i = threadIdx.x; i < nr * st; i += blockDim.x) {
    const int r = i / st, sl = i % st;
    dst[i] = tile_buf[r * (st + 1) + sl];
  }
  if (max_bits)
    for (int i = threadIdx.x; i < st; i += blockDim.x)
      if (smax[i]) atomicMax(&max_bits[t * st + i], smax[i]);
}

__global__ void __launch_bounds__(kConvThreads) to_natural_kernel(
    const float* __restrict__ in, float* __restrict__ nat, const int32_t* __restrict__ inv,
    int64_t rows, int S, int st) {
  extern __shared__ float tile_buf[];
  const int64_t h0 = (int64_t)blockIdx.x * kConvRows;
  const int t = blockIdx.y;
  const int nr = (int)min((int64_t)kConvRows, rows - h0);
  const float* src = in + ((size_t)t * rows + h0) * st;
  for (int i = threadIdx.x; i < nr * st; i += blockDim.x) {
    const int r = i / st, sl = i % st;
    tile_buf[r * (st + 1) + sl] = src[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kConvRows * st; i += blockDim.x) {
    const int sl = i / kConvRows, r = i % kConvRows;
    const int s = t * st + sl;
    if (r < nr && s < S) nat[(size_t)s * rows + inv[h0 + r]] = tile_buf[r * (st + 1) + sl];
  }
}

// ---------------------------------------------------------------------------
// CGLS vector updates.  Grid (kVecBlocks, ntiles); a thread visits elements
// i = tid*W + k*stride of its tile; stride is a multiple of st, so each thread
// always touches the same W slices and keeps their sums in registers.
// Per-block partial sums are reduced in a fixed order (deterministic).
// ---------------------------------------------------------------------------

template <int W>
__device__ void block_slice_sums(const FF* part, const uint32_t* pmax, int st, int tile,
                                 double* out_part, uint32_t* out_max, int nbx) {
  // part[W], pmax[W] per thread -> per-slice block totals
  __shared__ FF sd[kVecThreads * 4];
  __shared__ uint32_t sm[kVecThreads * 4];
  for (int w = 0; w < W; ++w) {
    sd[threadIdx.x * W + w] = part ? part[w] : FF{0.0f, 0.0f};
    sm[threadIdx.x * W + w] = pmax ? pmax[w] : 0u;
  }
  __syncthreads();
  const int per = st / W;  // threads sharing a slice set repeat every `per`
  for (int sl = threadIdx.x; sl < st; sl += blockDim.x) {
    const int t0 = sl / W, w = sl % W;
    FF acc{0.0f, 0.0f};
    uint32_t mx = 0;
    for (int t = t0; t < (int)blockDim.x; t += per) {
      acc = ff_add(acc, sd[t * W + w]);
      mx = max(mx, sm[t * W + w]);
    }
    const int gs = tile * st + sl;
    if (out_part) out_part[(size_t)gs * nbx + blockIdx.x] = ff_to_double(acc);
    if (out_max && mx) atomicMax(&out_max[gs], mx);
  }
  __syncthreads();
}

// W consecutive floats (one 16-byte access for W = 4: element offsets are
// multiples of 4 and every tile starts on a 16-byte boundary)
template <int W>
__device__ __forceinline__ void ldw(const float* p, float (&v)[W]) {
  if constexpr (W == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = p[w];
  }
}
template <int W>
__device__ __forceinline__ void stw(float* p, const float (&v)[W]) {
  if constexpr (W == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) p[w] = v[w];
  }
}

// x += alpha p (image); r -= alpha q (sinogram); max |r|, ||r||^2 partials
template <int W>
__global__ void __launch_bounds__(kVecThreads) update_xr_kernel(
    float* __restrict__ x, const float* __restrict__ p, int64_t npix_len,
    float* __restrict__ r, const float* __restrict__ q, int64_t nray_len, int st,
    const double* __restrict__ alpha, uint32_t* __restrict__ max_r, double* __restrict__ rpart) {
  const int tile = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * W;
  const int64_t start = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * W;
  const int sl0 = (int)(start % st);
  float a[W];
#pragma unroll
  for (int w = 0; w < W; ++w) a[w] = (float)alpha[tile * st + sl0 + w];
  float* xt = x + (size_t)tile * npix_len;
  const float* pt = p + (size_t)tile * npix_len;
  for (int64_t i = start; i < npix_len; i += stride) {
    float xv[W], pv[W];
    ldw<W>(xt + i, xv);
    ldw<W>(pt + i, pv);
#pragma unroll
    for (int w = 0; w < W; ++w) xv[w] = fmaf(a[w], pv[w], xv[w]);
    stw<W>(xt + i, xv);
  }
  float* rt = r + (size_t)tile * nray_len;
  const float* qt = q + (size_t)tile * nray_len;
  FF ss[W];
  uint32_t mx[W];
#pragma unroll
  for (int w = 0; w < W; ++w) { ss[w] = FF{0.0f, 0.0f}; mx[w] = 0u; }
  for (int64_t i = start; i < nray_len; i += stride) {
    float rv[W], qv[W];
    ldw<W>(rt + i, rv);
    ldw<W>(qt + i, qv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      rv[w] = fmaf(-a[w], qv[w], rv[w]);
      ss[w] = ff_add(ss[w], ff_sq(rv[w]));
      mx[w] = max(mx[w], __float_as_uint(fabsf(rv[w])));
    }
    stw<W>(rt + i, rv);
  }
  block_slice_sums<W>(ss, mx, st, tile, rpart, max_r, gridDim.x);
}

// p = s + beta p; max |p|
template <int W>
__global__ void __launch_bounds__(kVecThreads) update_p_kernel(
    float* __restrict__ p, const float* __restrict__ s, int64_t npix_len, int st,
    const double* __restrict__ beta, uint32_t* __restrict__ max_p) {
  const int tile = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * W;
  const int64_t start = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * W;
  const int sl0 = (int)(start % st);
  float bt[W];
  uint32_t mx[W];
#pragma unroll
  for (int w = 0; w < W; ++w) { bt[w] = (float)beta[tile * st + sl0 + w]; mx[w] = 0u; }
  float* ptile = p + (size_t)tile * npix_len;
  const float* stile = s + (size_t)tile * npix_len;
  for (int64_t i = start; i < npix_len; i += stride) {
    float pv[W], sv[W];
    ldw<W>(ptile + i, pv);
    ldw<W>(stile + i, sv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      pv[w] = fmaf(bt[w], pv[w], sv[w]);
      mx[w] = max(mx[w], __float_as_uint(fabsf(pv[w])));
    }
    stw<W>(ptile + i, pv);
  }
  block_slice_sums<W>(nullptr, mx, st, tile, nullptr, max_p, gridDim.x);
}

// r = r - q (x0 start) with max |r|; ||r||^2 partials of r (a = 0: only sums)
template <int W>
__global__ void __launch_bounds__(kVecThreads) residual_kernel(
    float* __restrict__ r, const float* __restrict__ q, int64_t nray_len, int st,
    uint32_t* __restrict__ max_r, double* __restrict__ rpart) {
  const int tile = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * W;
  const int64_t start = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * W;
  float* rt = r + (size_t)tile * nray_len;
  const float* qt = q ? q + (size_t)tile * nray_len : nullptr;
  FF ss[W];
  uint32_t mx[W];
#pragma unroll
  for (int w = 0; w < W; ++w) { ss[w] = FF{0.0f, 0.0f}; mx[w] = 0u; }
  for (int64_t i = start; i < nray_len; i += stride) {
    float rv[W];
    ldw<W>(rt + i, rv);
    if (qt) {
      float qv[W];
      ldw<W>(qt + i, qv);
#pragma unroll
      for (int w = 0; w < W; ++w) rv[w] = rv[w] - qv[w];
      stw<W>(rt + i, rv);
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
      ss[w] = ff_add(ss[w], ff_sq(rv[w]));
      mx[w] = max(mx[w], __float_as_uint(fabsf(rv[w])));
    }
  }
  block_slice_sums<W>(ss, mx, st, tile, rpart, max_r, gridDim.x);
}

// r = q - y (data-fit residual of the regularised reconstruction); max |r|,
// ||r||^2 partials
template <int W>
__global__ void __launch_bounds__(kVecThreads) sub_kernel(const float* __restrict__ q,
                                                          const float* __restrict__ y,
                                                          float* __restrict__ r, int64_t len, int st,
                                                          uint32_t* __restrict__ max_r,
                                                          double* __restrict__ rpart) {
  const int tile = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * W;
  const int64_t start = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * W;
  const float* qt = q + (size_t)tile * len;
  const float* yt = y + (size_t)tile * len;
  float* rt = r + (size_t)tile * len;
  FF ss[W];
  uint32_t mx[W];
#pragma unroll
  for (int w = 0; w < W; ++w) { ss[w] = FF{0.0f, 0.0f}; mx[w] = 0u; }
  for (int64_t i = start; i < len; i += stride) {
    float qv[W], yv[W], rv[W];
    ldw<W>(qt + i, qv);
    ldw<W>(yt + i, yv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      rv[w] = qv[w] - yv[w];
      ss[w] = ff_add(ss[w], ff_sq(rv[w]));
      mx[w] = max(mx[w], __float_as_uint(fabsf(rv[w])));
    }
    stw<W>(rt + i, rv);
  }
  block_slice_sums<W>(ss, mx, st, tile, rpart, max_r, gridDim.x);
}

// loss = sum over slices s < S of 0.5 ||r_s||^2 + tv[s]  (one block)
__global__ void loss_kernel(const double* __restrict__ rpart, int nbr, const double* __restrict__ tv,
                            int S, double* __restrict__ out) {
  __shared__ double sh[kVecThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < S * nbr; i += blockDim.x) a += 0.5 * rpart[i];
  for (int i = threadIdx.x; i < S; i += blockDim.x) a += tv[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ---------------------------------------------------------------------------
// scalars: one block per slice, fixed-order tree reduction of partials
// ---------------------------------------------------------------------------

__device__ double block_reduce_fixed(const double* part, int n) {
  __shared__ double sh[kVecThreads];
  // four independent accumulators per thread (loads and adds overlap),
  // combined in a fixed order
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int step = blockDim.x;
  int i = threadIdx.x;
  for (; i + 3 * step < n; i += 4 * step) {
    a0 += part[i];
    a1 += part[i + step];
    a2 += part[i + 2 * step];
    a3 += part[i + 3 * step];
  }
  for (; i < n; i += step) a0 += part[i];
  double a = (a0 + a1) + (a2 + a3);
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// after the initial back projection: gamma = ||s||^2, log[0]
__global__ void __launch_bounds__(kVecThreads) cgls_init_kernel(
    const double* gpart, int nbg, const double* rpart, int nbr, CglsScalars sc, double* log,
    int S_pad) {
  const int gs = blockIdx.x;
  const double g = block_reduce_fixed(gpart + (size_t)gs * nbg, nbg);
  const double rr = block_reduce_fixed(rpart + (size_t)gs * nbr, nbr);
  if (threadIdx.x == 0) {
    sc.gamma[gs] = g;
    const int act = g > 0.0;
    sc.active[gs] = act;
    sc.active0[gs] = act;
    sc.beta[gs] = 0.0;
    sc.max_p[gs] = 0u;
    if (log) {
      log[(size_t)gs * 2] = sqrt(rr);
      log[(size_t)gs * 2 + 1] = sqrt(g);
    }
  }
}

// delta = ||q||^2; alpha = gamma / delta (0 for a stopped slice)
__global__ void __launch_bounds__(kVecThreads) cgls_alpha_kernel(const double* dpart, int nbd,
                                                                 CglsScalars sc) {
  const int gs = blockIdx.x;
  const double d = block_reduce_fixed(dpart + (size_t)gs * nbd, nbd);
  if (threadIdx.x == 0) {
    int act = sc.active[gs] && d > 0.0;
    sc.active[gs] = act;
    sc.alpha[gs] = act ? sc.gamma[gs] / d : 0.0;
    sc.max_r[gs] = 0u;
  }
}

// gamma' = ||s||^2; beta = gamma'/gamma; log[k]
__global__ void __launch_bounds__(kVecThreads) cgls_beta_kernel(const double* gpart, int nbg,
                                                                const double* rpart, int nbr,
                                                                CglsScalars sc, double* log_k) {
  const int gs = blockIdx.x;
  const double g = block_reduce_fixed(gpart + (size_t)gs * nbg, nbg);
  const double rr = block_reduce_fixed(rpart + (size_t)gs * nbr, nbr);
  if (threadIdx.x == 0) {
    const int act = sc.active[gs];
    sc.beta[gs] = act ? g / sc.gamma[gs] : 0.0;
    if (act) sc.gamma[gs] = g;
    sc.active[gs] = act && g > 0.0;
    sc.max_p[gs] = 0u;
    if (log_k) {
      log_k[(size_t)gs * 2] = sqrt(rr);
      log_k[(size_t)gs * 2 + 1] = sqrt(g);
    }
  }
}

// resume from a saved state: gamma and the activity flags of the first S
// slices (padding slices inactive), log[0] from the residual partials
__global__ void __launch_bounds__(kVecThreads) cgls_restore_kernel(
    const double* gamma_in, const int32_t* active_in, int S, const double* rpart, int nbr,
    CglsScalars sc, double* log) {
  const int gs = blockIdx.x;
  const double rr = block_reduce_fixed(rpart + (size_t)gs * nbr, nbr);
  if (threadIdx.x == 0) {
    const double g = gs < S ? gamma_in[gs] : 0.0;
    const int act = gs < S ? active_in[gs] : 0;
    sc.gamma[gs] = g;
    sc.active[gs] = act;
    sc.active0[gs] = act;
    sc.beta[gs] = 0.0;
    if (log) {
      log[(size_t)gs * 2] = sqrt(rr);
      log[(size_t)gs * 2 + 1] = sqrt(g);
    }
  }
}

// save: gamma and the activity flags of the first S slices, and the header
__global__ void cgls_save_kernel(const CglsScalars sc, int S, CglsStateHeader hdr,
                                 CglsStateHeader* hdr_out, double* gamma_out, int32_t* active_out) {
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    gamma_out[s] = sc.gamma[s];
    active_out[s] = sc.active[s];
  }
  if (threadIdx.x == 0) *hdr_out = hdr;
}

inline unsigned conv_blocks(int64_t rows) { return (unsigned)((rows + kConvRows - 1) / kConvRows); }

}  // namespace

xct_status to_internal(const float* nat, float* in, const int32_t* inv_order, int64_t rows, int S,
                       int st, int ntiles, uint32_t* max_bits, cudaStream_t s) {
  if (st > 64) return XCT_ERR_UNSUPPORTED;
  dim3 grid(conv_blocks(rows), (unsigned)ntiles);
  size_t smem = (size_t)kConvRows * (st + 1) * sizeof(float);
  to_internal_kernel<<<grid, kConvThreads, smem, s>>>(nat, in, inv_order, rows, S, st, max_bits);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status to_natural(const float* in, float* nat, const int32_t* inv_order, int64_t rows, int S,
                      int st, int ntiles, cudaStream_t s) {
  dim3 grid(conv_blocks(rows), (unsigned)ntiles);
  size_t smem = (size_t)kConvRows * (st + 1) * sizeof(float);
  to_natural_kernel<<<grid, kConvThreads, smem, s>>>(in, nat, inv_order, rows, S, st);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

#define XCT_VEC_LAUNCH(KERNEL, ...)                                                   \
  do {                                                                                \
    dim3 grid_(kVecBlocks, (unsigned)ntiles);                                         \
    if (st % 4 == 0) KERNEL<4><<<grid_, kVecThreads, 0, s>>>(__VA_ARGS__);            \
    else KERNEL<1><<<grid_, kVecThreads, 0, s>>>(__VA_ARGS__);                        \
    count_launch();                                                                   \
    XCT_TRY_CUDA(cudaGetLastError());                                                 \
  } while (0)

xct_status cgls_update_xr(float* x, const float* p, int64_t npix, float* r, const float* q,
                          int64_t nray, int st, int ntiles, const CglsScalars& sc, double* rpart,
                          cudaStream_t s) {
  XCT_VEC_LAUNCH(update_xr_kernel, x, p, npix * st, r, q, nray * st, st, sc.alpha, sc.max_r, rpart);
  return XCT_OK;
}

xct_status cgls_update_p(float* p, const float* sv, int64_t npix, int st, int ntiles,
                         const CglsScalars& sc, cudaStream_t s) {
  XCT_VEC_LAUNCH(update_p_kernel, p, sv, npix * st, st, sc.beta, sc.max_p);
  return XCT_OK;
}

xct_status cgls_residual(float* r, const float* q, int64_t nray, int st, int ntiles,
                         uint32_t* max_r, double* rpart, cudaStream_t s) {
  XCT_VEC_LAUNCH(residual_kernel, r, q, nray * st, st, max_r, rpart);
  return XCT_OK;
}

xct_status vec_sub_sumsq(const float* q, const float* y, float* r, int64_t rows, int st,
                         int ntiles, uint32_t* max_r, double* rpart, cudaStream_t s) {
  XCT_VEC_LAUNCH(sub_kernel, q, y, r, rows * st, st, max_r, rpart);
  return XCT_OK;
}

xct_status vec_loss(const double* rpart, const double* tv, int S, double* out, cudaStream_t s) {
  loss_kernel<<<1, kVecThreads, 0, s>>>(rpart, kVecBlocks, tv, S, out);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status cgls_init_scalars(const double* gpart, int nbg, const double* rpart,
                             const CglsScalars& sc, double* log, int S_pad, cudaStream_t s) {
  cgls_init_kernel<<<S_pad, kVecThreads, 0, s>>>(gpart, nbg, rpart, kVecBlocks, sc, log, S_pad);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status cgls_alpha(const double* dpart, int nbd, const CglsScalars& sc, int S_pad,
                      cudaStream_t s) {
  cgls_alpha_kernel<<<S_pad, kVecThreads, 0, s>>>(dpart, nbd, sc);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status cgls_beta(const double* gpart, int nbg, const double* rpart, const CglsScalars& sc,
                     double* log_k, int S_pad, cudaStream_t s) {
  cgls_beta_kernel<<<S_pad, kVecThreads, 0, s>>>(gpart, nbg, rpart, kVecBlocks, sc, log_k);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status cgls_restore(const double* gamma_in, const int32_t* active_in, int S,
                        const double* rpart, const CglsScalars& sc, double* log, int S_pad,
                        cudaStream_t s) {
  cgls_restore_kernel<<<S_pad, kVecThreads, 0, s>>>(gamma_in, active_in, S, rpart, kVecBlocks, sc,
                                                     log);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

xct_status cgls_save(const CglsScalars& sc, int S, const CglsStateHeader& hdr,
                     CglsStateHeader* hdr_out, double* gamma_out, int32_t* active_out,
                     cudaStream_t s) {
  cgls_save_kernel<<<1, 256, 0, s>>>(sc, S, hdr, hdr_out, gamma_out, active_out);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

}  // namespace xct

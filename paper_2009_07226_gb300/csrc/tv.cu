// Regularised reconstruction support (Eq. 1 with R(x) = lambda * TV_eps(x)):
// a fused smoothed-total-variation value + gradient kernel, and a fused Adam
// update for the gradient iteration of Sec. II-A (forward project, residual,
// back project, update).
//
// TV_eps(x_s) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2) per slice, forward
// differences dx = x[i][j+1] - x[i][j], dy = x[i+1][j] - x[i][j], a difference
// past the last column / row taken as 0.  The gradient at (i, j) collects the
// three terms whose magnitude depends on x[i][j]:
//   -(dx + dy)/mag at (i, j),  dx/mag at (i, j-1),  dy/mag at (i-1, j).
#include <math.h>

#include "ff.cuh"
#include "xct_internal.cuh"

namespace xct {
namespace {

constexpr int kTvTile = 16;               // 16 x 16 pixels per block
constexpr int kTvThreads = kTvTile * kTvTile;

struct TvTerm {
  float dx, dy, mag;
};

__device__ __forceinline__ TvTerm tv_term(const float* xs, int n, int i, int j, float eps2) {
  const float c = xs[(size_t)i * n + j];
  const float dx = (j + 1 < n) ? xs[(size_t)i * n + j + 1] - c : 0.0f;
  const float dy = (i + 1 < n) ? xs[(size_t)(i + 1) * n + j] - c : 0.0f;
  return TvTerm{dx, dy, sqrtf(dx * dx + dy * dy + eps2)};
}

// grid (tiles_x * tiles_y, S); partial[s][tile] = sum of magnitudes (FP64
// value of an FP32-pair sum)
__global__ void __launch_bounds__(kTvThreads) tv_kernel(const float* __restrict__ x, int n, float eps,
                                                        float weight, float* __restrict__ grad,
                                                        int accumulate, double* __restrict__ partial) {
  __shared__ FF red[kTvThreads / 32];
  const int s = blockIdx.y;
  const int tiles_x = (n + kTvTile - 1) / kTvTile;
  const int ti = blockIdx.x / tiles_x, tj = blockIdx.x % tiles_x;
  const int i = ti * kTvTile + threadIdx.x / kTvTile;
  const int j = tj * kTvTile + threadIdx.x % kTvTile;
  const float* xs = x + (size_t)s * n * n;
  const float eps2 = eps * eps;
  FF val{0.0f, 0.0f};
  if (i < n && j < n) {
    const TvTerm t = tv_term(xs, n, i, j, eps2);
    val.hi = t.mag;
    float g = -(t.dx + t.dy) / t.mag;
    if (j > 0) {
      const TvTerm l = tv_term(xs, n, i, j - 1, eps2);
      g += l.dx / l.mag;
    }
    if (i > 0) {
      const TvTerm u = tv_term(xs, n, i - 1, j, eps2);
      g += u.dy / u.mag;
    }
    if (grad) {
      float* gp = grad + (size_t)s * n * n + (size_t)i * n + j;
      *gp = accumulate ? *gp + weight * g : weight * g;
    }
  }
  // block sum in FP32 pairs (ff.cuh), one FP64 partial per block
  for (int o = 16; o > 0; o >>= 1) val = ff_add(val, ff_shfl_xor(val, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x == 0) {
    FF t = red[0];
    for (int w = 1; w < kTvThreads / 32; ++w) t = ff_add(t, red[w]);
    partial[(size_t)s * gridDim.x + blockIdx.x] = ff_to_double(t);
  }
}

// value[s] = weight * sum of the slice's partials (fixed order)
__global__ void tv_reduce_kernel(const double* __restrict__ partial, int nparts, double weight,
                                 double* __restrict__ value) {
  __shared__ double sh[256];
  const int s = blockIdx.x;
  double a = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) a += partial[(size_t)s * nparts + k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) value[s] = weight * sh[0];
}

// Adam (bias-corrected, no weight decay), in the operation order of the
// common reference implementation:
//   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
//   x -= (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// The weights 1 - b1, 1 - b2 and the bias corrections are formed in FP64 on
// the host and rounded once to FP32 (1.0f - 0.9f would carry the rounding
// of 0.9f into the weight).
__global__ void adam_kernel(float* __restrict__ x, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t count,
                            float b1, float om1, float b2, float om2, float eps, float step_size,
                            float bc2_sqrt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + om1 * gk;
    const float vk = b2 * v[k] + om2 * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float denom = sqrtf(vk) / bc2_sqrt + eps;
    x[k] = x[k] - step_size * (mk / denom);
  }
}

bool host_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace

xct_status tv_launch(const float* x, int n, int S, double eps, double weight, float* grad,
                     bool accumulate, double* partial, double* value_dev, cudaStream_t s) {
  const int tiles = ((n + kTvTile - 1) / kTvTile) * ((n + kTvTile - 1) / kTvTile);
  tv_kernel<<<dim3((unsigned)tiles, (unsigned)S), kTvThreads, 0, s>>>(x, n, (float)eps, (float)weight,
                                                                      grad, accumulate ? 1 : 0, partial);
  tv_reduce_kernel<<<S, 256, 0, s>>>(partial, tiles, weight, value_dev);
  count_launch(2);
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

int tv_partials(int n) { return ((n + kTvTile - 1) / kTvTile) * ((n + kTvTile - 1) / kTvTile); }

xct_status adam_launch(float* x, const float* g, float* m, float* v, int64_t count, double lr,
                       double beta1, double beta2, double eps, int step, cudaStream_t s) {
  const double bc1 = 1.0 - pow(beta1, (double)step);
  const double bc2 = 1.0 - pow(beta2, (double)step);
  int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  adam_kernel<<<blocks, 256, 0, s>>>(x, g, m, v, count, (float)beta1, (float)(1.0 - beta1),
                                     (float)beta2, (float)(1.0 - beta2), (float)eps,
                                     (float)(lr / bc1), (float)sqrt(bc2));
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

}  // namespace xct

using namespace xct;

extern "C" xct_status xct_tv(const float* x, int32_t n, int32_t S, double eps, double weight,
                             float* grad, double* value, void* stream) {
  if (n < 1 || S < 0 || !x || !(eps > 0.0) || !isfinite(eps) || !isfinite(weight)) {
    set_error("xct_tv: bad arguments (n = %d, S = %d, eps = %g)", n, S, eps);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  if (host_ptr(x) || (grad && host_ptr(grad))) {
    set_error("xct_tv: x and grad must be device pointers");
    return XCT_ERR_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(s);
  double *partial, *val_d;
  XCT_TRY(ar.get(&partial, (size_t)S * tv_partials(n)));
  XCT_TRY(ar.get(&val_d, (size_t)S));
  XCT_TRY(tv_launch(x, n, S, eps, weight, grad, false, partial, val_d, s));
  if (value) {
    const bool vh = host_ptr(value);
    XCT_TRY_CUDA(cudaMemcpyAsync(value, val_d, sizeof(double) * S,
                                 vh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (vh) XCT_TRY_CUDA(cudaStreamSynchronize(s));
  }
  return XCT_OK;
}

extern "C" xct_status xct_adam(float* x, const float* g, float* m, float* v, int64_t count,
                               double lr, double beta1, double beta2, double eps, int32_t step,
                               void* stream) {
  if (count < 0 || step < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0) || ((!x || !g || !m || !v) && count > 0)) {
    set_error("xct_adam: bad arguments");
    return XCT_ERR_INVALID;
  }
  if (count == 0) return XCT_OK;
  return adam_launch(x, g, m, v, count, lr, beta1, beta2, eps, step, static_cast<cudaStream_t>(stream));
}

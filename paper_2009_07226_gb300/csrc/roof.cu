// xct_roof_probe: measures, on the GPU it runs on, the core roofs of the
// product kernels (the rates that bound a sparse product with many slices,
// where the matrix stream from HBM is not the limit).
//
// The product's inner step, per matrix entry and lane group, is: take a row
// index, read one 16-byte vector of a staged row from shared memory, and
// multiply-add it into the lane's accumulators (8 slices of a binary16 row
// through the mixed-precision FMA, or 4 FP32 slices).  The probe repeats
// exactly that step with row indices from a per-group linear congruential
// sequence (so 8 lanes read one contiguous 128-byte row, as in the product)
// and no matrix stream at all:
//   kind 0: 16-byte shared-memory gather + 8 mixed FMAs (fma.rn.f32.f16)
//   kind 1: the 8 mixed FMAs alone, operands from registers
//   kind 2: 8 FP32 FMAs alone (fmaf), operands from registers
//   kind 3: the 16-byte shared-memory gathers alone (consumed by an XOR)
//   kind 4: 16-byte gather + 4 FP32 slices through packed FP32 FMAs
// Every thread does `iters` steps of 4 gathers; the caller times the launch
// with events on `stream` and divides the operation count written to *ops
// (FMAs for kinds 0-2 and 4, 16-byte loads for kind 3) by it.
#include "xct_internal.cuh"

namespace xct {
namespace {

constexpr int kProbeThreads = 512;       // 16 warps, as the product's consumers
constexpr int kProbeRows = 256;          // staged rows of 128 bytes (32 KB)
__device__ float g_roof_sink;            // keeps the probe's results live

__device__ __forceinline__ void mixed8(float* acc, const uint4& v, unsigned short w) {
  const uint32_t* x = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const unsigned short lo = (unsigned short)(x[e] & 0xffffu), hi = (unsigned short)(x[e] >> 16);
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e]) : "h"(lo), "h"(w));
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e + 1]) : "h"(hi), "h"(w));
  }
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 2) roof_kernel(int64_t iters, uint32_t seed) {
  __shared__ uint4 rows[kProbeRows * 8];
  const int tid = threadIdx.x, lane = tid & 31, sub = lane & 7;
  // finite binary16 / FP32 bit patterns of moderate size
  for (int i = tid; i < kProbeRows * 8; i += blockDim.x) {
    const uint32_t h = 0x3000u | ((uint32_t)i * 37u & 0x3ffu);
    rows[i] = make_uint4(h | (h << 16), h | (h << 16), h | (h << 16), h | (h << 16));
  }
  __syncthreads();
  // one index sequence per group of 8 lanes (the lanes that share a row)
  uint32_t r = seed ^ ((uint32_t)(blockIdx.x * (kProbeThreads / 8) + (tid >> 3)) * 2654435761u);
  const unsigned short w = (unsigned short)(0x3800u | (r & 0xffu));
  float acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 0.0f;
  uint4 reg = make_uint4(0x30003000u + tid, 0x30013001u, 0x30023002u, 0x30033003u);
  uint32_t xo = 0;
  for (int64_t it = 0; it < iters; ++it) {
    uint4 xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      r = r * 1664525u + 1013904223u;
      if constexpr (KIND == 0 || KIND == 3 || KIND == 4)
        xv[q] = rows[(r >> 24) * 8 + sub];
      else
        xv[q] = make_uint4(reg.x ^ (r >> 24), reg.y, reg.z, reg.w);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (KIND == 0 || KIND == 1) {
        mixed8(acc, xv[q], w);
      } else if constexpr (KIND == 2) {
        const float* f = reinterpret_cast<const float*>(&xv[q]);
        const float wf = __uint_as_float(0x3f000000u | w);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] = fmaf(wf, f[e & 3], acc[e]);
      } else if constexpr (KIND == 3) {
        xo ^= xv[q].x ^ xv[q].y ^ xv[q].z ^ xv[q].w;
      } else {
        const float* f = reinterpret_cast<const float*>(&xv[q]);
        const float wf = __uint_as_float(0x3f000000u | w);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float2 c = make_float2(acc[2 * e], acc[2 * e + 1]);
          c = __ffma2_rn(make_float2(wf, wf), make_float2(f[2 * e], f[2 * e + 1]), c);
          acc[2 * e] = c.x;
          acc[2 * e + 1] = c.y;
        }
      }
    }
  }
  float s = __uint_as_float(xo & 0x007fffffu);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  // a comparison with a launch argument keeps every result (and load) live;
  // when it holds, the store is a harmless write of one scalar
  if (s == __uint_as_float(seed)) g_roof_sink = s;
}

}  // namespace
}  // namespace xct

extern "C" xct_status xct_roof_probe(int32_t kind, int64_t iters, int32_t ctas_per_sm,
                                     double* ops, void* stream) {
  using namespace xct;
  Trace trace_("xct_roof_probe");
  if (kind < 0 || kind > 4 || iters < 1 || iters > ((int64_t)1 << 40) || ctas_per_sm < 1 ||
      ctas_per_sm > 4 || !ops) {
    set_error("xct_roof_probe: bad arguments (kind %d, iters %lld, ctas_per_sm %d)", kind,
              (long long)iters, ctas_per_sm);
    return XCT_ERR_INVALID;
  }
  int dev = 0, sms = 0;
  XCT_TRY_CUDA(cudaGetDevice(&dev));
  XCT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * ctas_per_sm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t seed = 0x9e3779b9u;
  switch (kind) {
    case 0: roof_kernel<0><<<grid, kProbeThreads, 0, s>>>(iters, seed); break;
    case 1: roof_kernel<1><<<grid, kProbeThreads, 0, s>>>(iters, seed); break;
    case 2: roof_kernel<2><<<grid, kProbeThreads, 0, s>>>(iters, seed); break;
    case 3: roof_kernel<3><<<grid, kProbeThreads, 0, s>>>(iters, seed); break;
    default: roof_kernel<4><<<grid, kProbeThreads, 0, s>>>(iters, seed); break;
  }
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  const double threads = (double)grid * kProbeThreads;
  // per step and thread: 4 gathers of 16 bytes; FMAs: 4 x 8 (kinds 0-2), 4 x 4 (kind 4)
  const double per = kind == 3 ? 4.0 : (kind == 4 ? 16.0 : 32.0);
  *ops = threads * (double)iters * per;
  return XCT_OK;
}

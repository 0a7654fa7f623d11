// Exclusive prefix sums for plan construction (row pointers, tile offsets,
// footprint and stage offsets).  Three passes: per-tile totals, a
// sequential-carry scan of the totals by one block, per-tile rescans.
#include "xct_internal.cuh"

namespace xct {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ int64_t block_inclusive_scan(int64_t v, int64_t* warp_tot) {
  // warp-level inclusive scan
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += warp_tot[warp - 1];
  return v;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_totals(const T* in, int64_t n,
                                                                 int64_t* totals) {
  __shared__ int64_t red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) acc += (int64_t)in[idx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    totals[blockIdx.x] = t;
  }
}

// one block: exclusive scan of `totals` in place, carry across chunks
__global__ void __launch_bounds__(kScanThreads) scan_totals(int64_t* totals, int64_t nt) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nt; base += kScanThreads) {
    int64_t idx = base + threadIdx.x;
    int64_t v = idx < nt ? totals[idx] : 0;
    int64_t inc = block_inclusive_scan<int64_t>(v, warp_tot);
    int64_t c = carry;
    if (idx < nt) totals[idx] = c + inc - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c + inc;
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const T* in, int64_t n,
                                                           const int64_t* tile_off, int64_t* out) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? (int64_t)in[idx] : 0;
    sum += v[i];
  }
  int64_t inc = block_inclusive_scan<int64_t>(sum, warp_tot);
  int64_t run = tile_off[blockIdx.x] + inc - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
    if (idx == n - 1) out[n] = run;
  }
}

__global__ void write_zero_total(int64_t* out) { out[0] = 0; }

template <class T>
xct_status exclusive_scan(const T* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    write_zero_total<<<1, 1, 0, s>>>(out);
    count_launch();
    XCT_TRY_CUDA(cudaGetLastError());
    return XCT_OK;
  }
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  int64_t* totals = static_cast<int64_t*>(dalloc(sizeof(int64_t) * nt, s));
  if (!totals) return XCT_ERR_OOM;
  scan_tile_totals<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, totals);
  scan_totals<<<1, kScanThreads, 0, s>>>(totals, nt);
  scan_tiles<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, totals, out);
  count_launch(3);
  cudaError_t e = cudaGetLastError();
  dfree(totals, sizeof(int64_t) * nt, s);
  if (e != cudaSuccess) {
    set_error("scan launch failed: %s", cudaGetErrorString(e));
    return XCT_ERR_CUDA;
  }
  return XCT_OK;
}

}  // namespace

xct_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return exclusive_scan<int32_t>(in, out, n, s);
}
xct_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return exclusive_scan<int64_t>(in, out, n, s);
}

}  // namespace xct

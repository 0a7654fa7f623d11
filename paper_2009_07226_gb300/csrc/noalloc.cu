// xct_project_noalloc: the projection of xct_project with every piece of
// working memory taken from one fixed, file-scope device array instead of the
// allocator.
//
// Some callers cannot allocate device memory while they run: a process whose
// device memory is owned up front by another component (a serving runtime or
// a framework's caching allocator that has reserved the whole budget and
// rejects foreign allocations), or a latency-critical loop (for example one
// that reconstructs detector frames as they stream in) where an allocation
// could block or fail at an unpredictable moment.  For them this entry point
// touches only memory that exists before the call: the plan, the caller's
// buffers and the array below.
//
// The array holds kNoAllocBytes (32 MiB) per GPU.  CUDA loads a module's
// device variables with the module, and by default (lazy loading) a module is
// loaded on its first use; this file has no kernels, so its first use is the
// address lookup.  xct_plan therefore looks the address up on the plan's
// device (noalloc_reserve): from then on the array is resident on that device
// until the process exits, and a no-allocation call finds it in place.  Its
// host-side name is only a stand-in for the device symbol, so the device
// address comes from cudaGetSymbolAddress, made with the device current, and
// is cached per device.  All calls share the array and it keeps the last
// call's contents: everything that must start at zero is cleared by each
// call, and calls whose GPU work overlaps (several streams, several host
// threads) race on it.
#include <mutex>

#include "xct_internal.cuh"

namespace xct {
namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Makes `dev` current for its lifetime and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  xct_status enter(int dev) {
    XCT_TRY_CUDA(cudaGetDevice(&prev));
    if (prev != dev) XCT_TRY_CUDA(cudaSetDevice(dev));
    return XCT_OK;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// The array's address on `dev`, which must be the current device.
xct_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return XCT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the fixed scratch array failed: %s", cudaGetErrorString(e));
      return XCT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return XCT_OK;
}

bool device_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

xct_status noalloc_reserve(int device) {
  DeviceGuard g;
  XCT_TRY(g.enter(device));
  void* p = nullptr;
  return scratch_address(device, &p);
}

}  // namespace xct

extern "C" xct_status xct_project_noalloc(xct_plan_t plan, const float* x, float* y, int32_t S,
                                          void* stream) {
  using namespace xct;
  Trace trace_("xct_project_noalloc");
  if (!plan) {
    set_error("plan is NULL");
    return XCT_ERR_INVALID;
  }
  if (S < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  Plan& p = *static_cast<Plan*>(plan);
  // the plan's matrices, the array and the launches all on the plan's device
  DeviceGuard dg;
  XCT_TRY(dg.enter(p.device));
  if (!device_accessible(x) || !device_accessible(y)) {
    set_error("xct_project_noalloc takes device pointers only (host buffers would need staging)");
    return XCT_ERR_INVALID;
  }
  const Layout& L = p.la;
  const int st = pick_slices_per_tile(p.storage, S);
  const int ntiles = (S + st - 1) / st;
  const size_t S_pad = (size_t)st * ntiles;
  // carve the fixed array: internal input, internal output, 16-bit staging
  // copy, per-slice maxima, work counter
  const size_t b_xi = align256(sizeof(float) * (size_t)L.ncols * S_pad);
  const size_t b_yi = align256(sizeof(float) * (size_t)L.nrows * S_pad);
  const size_t b_h = stages16(p.storage) ? align256(sizeof(uint16_t) * (size_t)L.ncols * S_pad) : 0;
  const size_t b_mx = align256(sizeof(uint32_t) * S_pad);
  const size_t b_w = 256;
  const size_t need = b_xi + b_yi + b_h + b_mx + b_w;
  if (need > kNoAllocBytes) {
    set_error("xct_project_noalloc needs %zu bytes of working memory for S = %d on this plan; "
              "the fixed array holds %zu (use xct_project, or fewer slices per call)",
              need, S, kNoAllocBytes);
    return XCT_ERR_INVALID;
  }
  void* base = nullptr;
  XCT_TRY(scratch_address(p.device, &base));
  unsigned char* b = static_cast<unsigned char*>(base);
  float* Xi = reinterpret_cast<float*>(b);
  float* Yi = reinterpret_cast<float*>(b + b_xi);
  uint16_t* h16 = b_h ? reinterpret_cast<uint16_t*>(b + b_xi + b_yi) : nullptr;
  uint32_t* mx = reinterpret_cast<uint32_t*>(b + b_xi + b_yi + b_h);
  int* work = reinterpret_cast<int*>(b + b_xi + b_yi + b_h + b_mx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the maxima accumulate with atomicMax: they must start at zero every call
  XCT_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(uint32_t) * S_pad, s));
  XCT_TRY(to_internal(x, Xi, p.pix_inv, L.ncols, S, st, ntiles, mx, s));
  SpmmArgs a{&L, Xi, Yi, st, ntiles, p.storage, p.mat_scale_exp, mx, nullptr, h16, work, p.err};
  XCT_TRY(spmm(a, s));
  XCT_TRY(to_natural(Yi, y, p.ray_inv, L.nrows, S, st, ntiles, s));
  return XCT_OK;
}

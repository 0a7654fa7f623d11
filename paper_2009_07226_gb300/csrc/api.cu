// C-ABI entry points of libxct.so (declared in include/xct.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <memory>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "xct_internal.cuh"
#include "xct_vec.cuh"

namespace xct {

// ---------------------------------------------------------------------------
// errors, allocation hook, launch count
// ---------------------------------------------------------------------------

static thread_local char g_err[1024] = "";
std::atomic<int64_t> g_launches{0};
std::atomic<uint64_t> g_wait_ns{2000000000ull};
uint64_t wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {
struct AllocHook {
  xct_alloc_fn alloc = nullptr;
  xct_free_fn release = nullptr;
  void* ctx = nullptr;
};
std::mutex g_hook_mu;
AllocHook g_hook;

AllocHook hook() {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  return g_hook;
}
}  // namespace

void* dalloc(size_t bytes, cudaStream_t s) {
  AllocHook h = hook();
  if (h.alloc) {
    void* p = h.alloc(bytes, (void*)s, h.ctx);
    if (!p) set_error("allocator callback failed for %zu bytes", bytes);
    return p;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return nullptr;
  }
  return p;
}

void dfree(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  AllocHook h = hook();
  if (h.release) {
    h.release(p, bytes, (void*)s, h.ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

namespace {

bool is_host_pointer(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// A vector argument that may live on the host: a device view of it.
template <class T>
struct DevViewT {
  T* dev = nullptr;
  bool host = false;
};
using DevView = DevViewT<float>;

template <class T>
xct_status device_view(const T* user, size_t count, bool copy_in, Arena& ar, cudaStream_t s,
                       DevViewT<T>& v) {
  v.host = is_host_pointer(user);
  if (!v.host) {
    v.dev = const_cast<T*>(user);
    return XCT_OK;
  }
  XCT_TRY(ar.get(&v.dev, count));
  if (copy_in && count)
    XCT_TRY_CUDA(cudaMemcpyAsync(v.dev, user, count * sizeof(T), cudaMemcpyHostToDevice, s));
  return XCT_OK;
}

xct_status check_plan(xct_plan_t plan) {
  if (!plan) {
    set_error("plan is NULL");
    return XCT_ERR_INVALID;
  }
  return XCT_OK;
}

// Per-phase CUDA-event timing (XCT_CGLS_TIMING).
struct PhaseTimer {
  cudaStream_t s = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  cudaEvent_t cur = nullptr;
  xct_status begin(int kind) {
    (void)kind;
    XCT_TRY_CUDA(cudaEventCreate(&cur));
    XCT_TRY_CUDA(cudaEventRecord(cur, s));
    return XCT_OK;
  }
  xct_status end(int kind) {
    cudaEvent_t e;
    XCT_TRY_CUDA(cudaEventCreate(&e));
    XCT_TRY_CUDA(cudaEventRecord(e, s));
    ev.push_back({kind, {cur, e}});
    cur = nullptr;
    return XCT_OK;
  }
  ~PhaseTimer() {
    for (auto& x : ev) {
      cudaEventDestroy(x.second.first);
      cudaEventDestroy(x.second.second);
    }
    if (cur) cudaEventDestroy(cur);
  }
};

struct CglsBufs {
  float *X, *R, *P, *Q, *Sv;
  uint16_t *h_pix, *h_ray;   // 16-bit staging copies of the product inputs
  int* work;                 // work counter of the persistent product
  double *dpart, *gpart, *rpart, *log;
  uint32_t* max_x;
  CglsScalars sc;
};

// A saved CGLS state in device memory (sections of one buffer; layout in
// xct_vec.cuh).
struct CglsState {
  CglsStateHeader* hdr = nullptr;
  double* gamma = nullptr;
  int32_t* active = nullptr;
  float *x = nullptr, *r = nullptr, *p = nullptr;
};

size_t state_bytes(int64_t npix, int64_t nray, int S) {
  const size_t act = ((size_t)S * 4 + 7) / 8 * 8;
  return sizeof(CglsStateHeader) + (size_t)S * 8 + act + (size_t)S * (2 * npix + nray) * 4;
}

CglsState state_view(unsigned char* base, int64_t npix, int64_t nray, int S) {
  CglsState v;
  size_t o = 0;
  v.hdr = reinterpret_cast<CglsStateHeader*>(base);
  o += sizeof(CglsStateHeader);
  v.gamma = reinterpret_cast<double*>(base + o);
  o += (size_t)S * 8;
  v.active = reinterpret_cast<int32_t*>(base + o);
  o += ((size_t)S * 4 + 7) / 8 * 8;
  v.x = reinterpret_cast<float*>(base + o);
  o += (size_t)S * npix * 4;
  v.r = reinterpret_cast<float*>(base + o);
  o += (size_t)S * nray * 4;
  v.p = reinterpret_cast<float*>(base + o);
  return v;
}

// timed phases: projection (0), back projection (1), 16-bit staging of a
// product input (2), vector updates (3), FP64 scalars (4)
constexpr int kPhProject = 0, kPhBackproject = 1, kPhStage = 2, kPhVector = 3, kPhScalar = 4;

xct_status spmm_timed(const SpmmArgs& a, int kind, PhaseTimer* tm, cudaStream_t s) {
  if (tm) XCT_TRY(tm->begin(kPhStage));
  XCT_TRY(spmm_stage(a, s));
  if (tm) XCT_TRY(tm->end(kPhStage));
  if (tm) XCT_TRY(tm->begin(kind));
  XCT_TRY(spmm_run(a, s));
  if (tm) XCT_TRY(tm->end(kind));
  return XCT_OK;
}

// Enqueue the whole solve on stream s (graph-capturable: no host syncs).
xct_status enqueue_cgls(Plan& p, const float* yd, float* xd, int S, int st, int ntiles, int iters,
                        bool x0, CglsBufs& B, cudaStream_t s, PhaseTimer* tm,
                        const CglsState* resume = nullptr, const CglsState* save = nullptr,
                        int iters_before = 0) {
  const int S_pad = st * ntiles;
  const int64_t npix = p.npix, nray = p.nray;
  const int k = p.mat_scale_exp;
  const SpmmArgs probe_at{&p.lat, B.R, B.Sv, st, ntiles, p.storage, k, B.sc.max_r, B.gpart,
                          B.h_ray, B.work, p.err};
  const int nb_at = spmm_dot_count(probe_at);
  if (resume) {
    // x, r, p and the scalars of the saved iteration; its log entry
    XCT_TRY_CUDA(cudaMemsetAsync(B.max_x, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(to_internal(resume->x, B.X, p.pix_inv, npix, S, st, ntiles, B.max_x, s));
    XCT_TRY_CUDA(cudaMemsetAsync(B.sc.max_p, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(to_internal(resume->p, B.P, p.pix_inv, npix, S, st, ntiles, B.sc.max_p, s));
    XCT_TRY_CUDA(cudaMemsetAsync(B.sc.max_r, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(to_internal(resume->r, B.R, p.ray_inv, nray, S, st, ntiles, B.sc.max_r, s));
    XCT_TRY_CUDA(cudaMemsetAsync(B.sc.max_r, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(cgls_residual(B.R, nullptr, nray, st, ntiles, B.sc.max_r, B.rpart, s));
    XCT_TRY(cgls_restore(resume->gamma, resume->active, S, B.rpart, B.sc, B.log, S_pad, s));
  } else {
    XCT_TRY_CUDA(cudaMemsetAsync(B.sc.max_r, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(to_internal(yd, B.R, p.ray_inv, nray, S, st, ntiles, B.sc.max_r, s));
    if (x0) {
      XCT_TRY_CUDA(cudaMemsetAsync(B.max_x, 0, sizeof(uint32_t) * S_pad, s));
      XCT_TRY(to_internal(xd, B.X, p.pix_inv, npix, S, st, ntiles, B.max_x, s));
      SpmmArgs a{&p.la, B.X, B.Q, st, ntiles, p.storage, k, B.max_x, nullptr, B.h_pix, B.work, p.err};
      XCT_TRY(spmm_timed(a, 0, tm, s));
      XCT_TRY_CUDA(cudaMemsetAsync(B.sc.max_r, 0, sizeof(uint32_t) * S_pad, s));
      XCT_TRY(cgls_residual(B.R, B.Q, nray, st, ntiles, B.sc.max_r, B.rpart, s));
    } else {
      XCT_TRY_CUDA(cudaMemsetAsync(B.X, 0, sizeof(float) * npix * S_pad, s));
      XCT_TRY(cgls_residual(B.R, nullptr, nray, st, ntiles, B.sc.max_r, B.rpart, s));
    }
    XCT_TRY_CUDA(cudaMemsetAsync(B.P, 0, sizeof(float) * npix * S_pad, s));
    {
      SpmmArgs a{&p.lat, B.R, B.Sv, st, ntiles, p.storage, k, B.sc.max_r, B.gpart, B.h_ray, B.work, p.err};
      XCT_TRY(spmm_timed(a, 1, tm, s));
    }
    if (tm) XCT_TRY(tm->begin(kPhScalar));
    XCT_TRY(cgls_init_scalars(B.gpart, nb_at, B.rpart, B.sc, B.log, S_pad, s));
    if (tm) XCT_TRY(tm->end(kPhScalar));
    if (tm) XCT_TRY(tm->begin(kPhVector));
    XCT_TRY(cgls_update_p(B.P, B.Sv, npix, st, ntiles, B.sc, s));
    if (tm) XCT_TRY(tm->end(kPhVector));
  }
  for (int it = 1; it <= iters; ++it) {
    SpmmArgs ap{&p.la, B.P, B.Q, st, ntiles, p.storage, k, B.sc.max_p, B.dpart, B.h_pix, B.work, p.err};
    XCT_TRY(spmm_timed(ap, 0, tm, s));
    if (tm) XCT_TRY(tm->begin(kPhScalar));
    XCT_TRY(cgls_alpha(B.dpart, spmm_dot_count(ap), B.sc, S_pad, s));
    if (tm) XCT_TRY(tm->end(kPhScalar));
    if (tm) XCT_TRY(tm->begin(kPhVector));
    XCT_TRY(cgls_update_xr(B.X, B.P, npix, B.R, B.Q, nray, st, ntiles, B.sc, B.rpart, s));
    if (tm) XCT_TRY(tm->end(kPhVector));
    SpmmArgs at{&p.lat, B.R, B.Sv, st, ntiles, p.storage, k, B.sc.max_r, B.gpart, B.h_ray, B.work, p.err};
    XCT_TRY(spmm_timed(at, 1, tm, s));
    if (tm) XCT_TRY(tm->begin(kPhScalar));
    XCT_TRY(cgls_beta(B.gpart, nb_at, B.rpart, B.sc, B.log + (size_t)it * S_pad * 2, S_pad, s));
    if (tm) XCT_TRY(tm->end(kPhScalar));
    if (tm) XCT_TRY(tm->begin(kPhVector));
    XCT_TRY(cgls_update_p(B.P, B.Sv, npix, st, ntiles, B.sc, s));
    if (tm) XCT_TRY(tm->end(kPhVector));
  }
  XCT_TRY(to_natural(B.X, xd, p.pix_inv, npix, S, st, ntiles, s));
  if (save) {
    XCT_TRY(to_natural(B.X, save->x, p.pix_inv, npix, S, st, ntiles, s));
    XCT_TRY(to_natural(B.R, save->r, p.ray_inv, nray, S, st, ntiles, s));
    XCT_TRY(to_natural(B.P, save->p, p.pix_inv, npix, S, st, ntiles, s));
    const CglsStateHeader hdr{kCglsStateMagic, S, iters_before + iters, npix, nray};
    XCT_TRY(cgls_save(B.sc, S, hdr, save->hdr, save->gamma, save->active, s));
  }
  return XCT_OK;
}

struct StreamGuard {
  cudaStream_t s = nullptr;
  ~StreamGuard() {
    if (s) cudaStreamDestroy(s);
  }
};
struct EventGuard {
  cudaEvent_t e = nullptr;
  ~EventGuard() {
    if (e) cudaEventDestroy(e);
  }
};
struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  ~GraphGuard() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

xct_status cgls_impl(Plan& p, const float* y, float* x, int32_t S, int32_t iters, uint32_t flags,
                     double* resid, void* state, cudaStream_t us) {
  const int st = pick_slices_per_tile(p.storage, S);
  const int ntiles = (S + st - 1) / st;
  const int S_pad = st * ntiles;
  Arena ar(us);
  DevView yv, xv, sv;
  const bool resume = (flags & XCT_CGLS_RESUME) != 0, save = (flags & XCT_CGLS_SAVE) != 0;
  XCT_TRY(device_view(y, (size_t)S * p.nray, !resume, ar, us, yv));
  const bool x0 = (flags & XCT_CGLS_X0) != 0;
  XCT_TRY(device_view(x, (size_t)S * p.npix, x0 && !resume, ar, us, xv));
  CglsState st_view{};
  int iters_before = 0;
  if (resume || save) {
    const size_t nbytes = state_bytes(p.npix, p.nray, S);
    XCT_TRY(device_view(static_cast<const float*>(state), nbytes / 4, resume, ar, us, sv));
    st_view = state_view(reinterpret_cast<unsigned char*>(sv.dev), p.npix, p.nray, S);
    if (resume) {
      CglsStateHeader h{};
      XCT_TRY_CUDA(cudaMemcpyAsync(&h, st_view.hdr, sizeof(h), cudaMemcpyDeviceToHost, us));
      XCT_TRY_CUDA(cudaStreamSynchronize(us));
      if (h.magic != kCglsStateMagic || h.S != S || h.npix != p.npix || h.nray != p.nray ||
          h.iters_done < 0) {
        set_error("the CGLS state does not belong to this plan and slice count");
        return XCT_ERR_INVALID;
      }
      iters_before = h.iters_done;
    }
  }
  const CglsState* resume_v = resume ? &st_view : nullptr;
  const CglsState* save_v = save ? &st_view : nullptr;
  CglsBufs B{};
  XCT_TRY(ar.get(&B.X, (size_t)p.npix * S_pad));
  XCT_TRY(ar.get(&B.P, (size_t)p.npix * S_pad));
  XCT_TRY(ar.get(&B.Sv, (size_t)p.npix * S_pad));
  XCT_TRY(ar.get(&B.R, (size_t)p.nray * S_pad));
  XCT_TRY(ar.get(&B.Q, (size_t)p.nray * S_pad));
  if (stages16(p.storage)) {
    XCT_TRY(ar.get(&B.h_pix, (size_t)p.npix * S_pad));
    XCT_TRY(ar.get(&B.h_ray, (size_t)p.nray * S_pad));
  }
  XCT_TRY(ar.get(&B.dpart, (size_t)S_pad * std::max(p.la.nblocks, 1)));
  XCT_TRY(ar.get(&B.gpart, (size_t)S_pad * std::max(p.lat.nblocks, 1)));
  XCT_TRY(ar.get(&B.work, 1));
  XCT_TRY(ar.get(&B.rpart, (size_t)S_pad * kVecBlocks));
  XCT_TRY(ar.get(&B.log, (size_t)(iters + 1) * S_pad * 2));
  XCT_TRY(ar.get(&B.max_x, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.gamma, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.alpha, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.beta, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.active, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.active0, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.max_r, (size_t)S_pad));
  XCT_TRY(ar.get(&B.sc.max_p, (size_t)S_pad));

  const bool timing = (flags & XCT_CGLS_TIMING) != 0;
  const bool graph = !(flags & (XCT_CGLS_NO_GRAPH | XCT_CGLS_TIMING));
  if (graph) {
    StreamGuard cs;
    EventGuard e0, e1;
    GraphGuard gg;
    XCT_TRY_CUDA(cudaStreamCreateWithFlags(&cs.s, cudaStreamNonBlocking));
    XCT_TRY_CUDA(cudaEventCreateWithFlags(&e0.e, cudaEventDisableTiming));
    XCT_TRY_CUDA(cudaEventCreateWithFlags(&e1.e, cudaEventDisableTiming));
    XCT_TRY_CUDA(cudaEventRecord(e0.e, us));
    XCT_TRY_CUDA(cudaStreamWaitEvent(cs.s, e0.e, 0));
    XCT_TRY_CUDA(cudaStreamBeginCapture(cs.s, cudaStreamCaptureModeThreadLocal));
    xct_status st_enq = enqueue_cgls(p, yv.dev, xv.dev, S, st, ntiles, iters, x0, B, cs.s, nullptr,
                                     resume_v, save_v, iters_before);
    cudaError_t ec = cudaStreamEndCapture(cs.s, &gg.g);
    if (st_enq != XCT_OK) return st_enq;
    if (ec != cudaSuccess) {
      set_error("graph capture failed: %s", cudaGetErrorString(ec));
      return XCT_ERR_CUDA;
    }
    XCT_TRY_CUDA(cudaGraphInstantiate(&gg.x, gg.g, 0));
    XCT_TRY_CUDA(cudaGraphLaunch(gg.x, cs.s));
    XCT_TRY_CUDA(cudaEventRecord(e1.e, cs.s));
    XCT_TRY_CUDA(cudaStreamWaitEvent(us, e1.e, 0));
    XCT_TRY_CUDA(cudaStreamSynchronize(cs.s));
  } else {
    PhaseTimer tm;
    tm.s = us;
    XCT_TRY(enqueue_cgls(p, yv.dev, xv.dev, S, st, ntiles, iters, x0, B, us,
                         timing ? &tm : nullptr, resume_v, save_v, iters_before));
    if (timing) {
      XCT_TRY_CUDA(cudaStreamSynchronize(us));
      double t[5] = {0, 0, 0, 0, 0};
      int64_t n[5] = {0, 0, 0, 0, 0};
      for (auto& e : tm.ev) {
        float ms = 0;
        XCT_TRY_CUDA(cudaEventElapsedTime(&ms, e.second.first, e.second.second));
        t[e.first] += ms;
        n[e.first] += 1;
      }
      p.stats.t_project_ms = t[kPhProject];
      p.stats.t_backproject_ms = t[kPhBackproject];
      p.stats.t_stage_ms = t[kPhStage];
      p.stats.t_vector_ms = t[kPhVector];
      p.stats.t_scalar_ms = t[kPhScalar];
      p.stats.t_other_ms = t[kPhStage] + t[kPhVector] + t[kPhScalar];
      p.stats.n_project = n[kPhProject];
      p.stats.n_backproject = n[kPhBackproject];
    }
  }
  if (resid) {
    const bool rh = is_host_pointer(resid);
    XCT_TRY_CUDA(cudaMemcpy2DAsync(resid, sizeof(double) * 2 * S, B.log, sizeof(double) * 2 * S_pad,
                                   sizeof(double) * 2 * S, iters + 1,
                                   rh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, us));
  }
  if (xv.host)
    XCT_TRY_CUDA(cudaMemcpyAsync(x, xv.dev, sizeof(float) * S * p.npix, cudaMemcpyDeviceToHost, us));
  if (save && sv.host)
    XCT_TRY_CUDA(cudaMemcpyAsync(state, sv.dev, state_bytes(p.npix, p.nray, S),
                                 cudaMemcpyDeviceToHost, us));
  std::vector<int> act0((size_t)S_pad);
  XCT_TRY_CUDA(cudaMemcpyAsync(act0.data(), B.sc.active0, sizeof(int) * S_pad,
                               cudaMemcpyDeviceToHost, us));
  int kerr = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&kerr, p.err, sizeof(int), cudaMemcpyDeviceToHost, us));
  XCT_TRY_CUDA(cudaStreamSynchronize(us));
  if (kerr) {
    XCT_TRY_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), us));
    set_error("a bounded wait in the product kernel ran out; results are invalid");
    return XCT_ERR_TIMEOUT;
  }
  bool any = false;
  for (int i = 0; i < S; ++i) any = any || act0[i];
  if (!any) {
    set_error("CGLS breakdown: every slice has A^T r_0 = 0");
    return XCT_ERR_BREAKDOWN;
  }
  return XCT_OK;
}

// The product kernel's bounded waits report through the plan's error flag.
xct_status check_kernel_flag(Plan& p, cudaStream_t s) {
  int kerr = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&kerr, p.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  if (kerr) {
    XCT_TRY_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), s));
    set_error("a bounded wait in the product kernel ran out; results are invalid");
    return XCT_ERR_TIMEOUT;
  }
  return XCT_OK;
}

// A copy stream that is drained before it is destroyed (declared after the
// arena whose buffers its copies use, so it goes first).
struct CopyStream {
  cudaStream_t s = nullptr;
  ~CopyStream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

// Host vectors and several slice tiles: the slice-tile pipeline.  Tile t+1's
// host-to-device copy and tile t-1's device-to-host copy run on two copy
// streams (one per direction, so neither waits behind the other) while tile
// t is packed, multiplied and unpacked on `s`, with two device buffers per
// vector (the single-GPU form of the paper's pipelined
// minibatches, whose transfers overlap the products, Sec. III-D).  Each
// tile is computed exactly as in the one-launch form, so the results are
// identical.
xct_status apply_pipelined(Plan& p, bool transposed, const float* in, float* out, int32_t S,
                           int st, int ntiles, bool in_host, bool out_host, cudaStream_t s) {
  const Layout& L = transposed ? p.lat : p.la;
  const int32_t* in_inv = transposed ? p.ray_inv : p.pix_inv;
  const int32_t* out_inv = transposed ? p.pix_inv : p.ray_inv;
  const int64_t nin = L.ncols, nout = L.nrows;
  Arena ar(s);
  float *Xn[2] = {nullptr, nullptr}, *Yn[2] = {nullptr, nullptr}, *Xi[2], *Yi[2];
  uint32_t* mx[2];
  uint16_t* h16[2] = {nullptr, nullptr};
  int* work;
  for (int b = 0; b < 2; ++b) {
    if (in_host) XCT_TRY(ar.get(&Xn[b], (size_t)nin * st));
    if (out_host) XCT_TRY(ar.get(&Yn[b], (size_t)nout * st));
    XCT_TRY(ar.get(&Xi[b], (size_t)nin * st));
    XCT_TRY(ar.get(&Yi[b], (size_t)nout * st));
    XCT_TRY(ar.get(&mx[b], (size_t)st));
    if (stages16(p.storage)) XCT_TRY(ar.get(&h16[b], (size_t)nin * st));
  }
  XCT_TRY(ar.get(&work, 1));
  CopyStream cin, cout;
  XCT_TRY_CUDA(cudaStreamCreateWithFlags(&cin.s, cudaStreamNonBlocking));
  XCT_TRY_CUDA(cudaStreamCreateWithFlags(&cout.s, cudaStreamNonBlocking));
  EventGuard ev_alloc, ev_in[2], ev_used[2], ev_out[2], ev_d2h[2];
  for (EventGuard* e : {&ev_alloc, &ev_in[0], &ev_in[1], &ev_used[0], &ev_used[1], &ev_out[0],
                        &ev_out[1], &ev_d2h[0], &ev_d2h[1]})
    XCT_TRY_CUDA(cudaEventCreateWithFlags(&e->e, cudaEventDisableTiming));
  // the buffers are stream-ordered allocations on s
  XCT_TRY_CUDA(cudaEventRecord(ev_alloc.e, s));
  XCT_TRY_CUDA(cudaStreamWaitEvent(cin.s, ev_alloc.e, 0));
  XCT_TRY_CUDA(cudaStreamWaitEvent(cout.s, ev_alloc.e, 0));
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const int St = S - t * st < st ? S - t * st : st;
    const float* xin = in + (size_t)t * st * nin;
    if (in_host) {
      if (t >= 2) XCT_TRY_CUDA(cudaStreamWaitEvent(cin.s, ev_used[b].e, 0));
      XCT_TRY_CUDA(cudaMemcpyAsync(Xn[b], xin, sizeof(float) * St * nin, cudaMemcpyHostToDevice,
                                   cin.s));
      XCT_TRY_CUDA(cudaEventRecord(ev_in[b].e, cin.s));
      XCT_TRY_CUDA(cudaStreamWaitEvent(s, ev_in[b].e, 0));
      xin = Xn[b];
    }
    XCT_TRY_CUDA(cudaMemsetAsync(mx[b], 0, sizeof(uint32_t) * st, s));
    XCT_TRY(to_internal(xin, Xi[b], in_inv, nin, St, st, 1, mx[b], s));
    if (in_host) XCT_TRY_CUDA(cudaEventRecord(ev_used[b].e, s));
    SpmmArgs a{&L, Xi[b], Yi[b], st, 1, p.storage, p.mat_scale_exp, mx[b], nullptr, h16[b], work,
               p.err};
    XCT_TRY(spmm(a, s));
    float* yout = out + (size_t)t * st * nout;
    if (out_host) {
      if (t >= 2) XCT_TRY_CUDA(cudaStreamWaitEvent(s, ev_d2h[b].e, 0));
      XCT_TRY(to_natural(Yi[b], Yn[b], out_inv, nout, St, st, 1, s));
      XCT_TRY_CUDA(cudaEventRecord(ev_out[b].e, s));
      XCT_TRY_CUDA(cudaStreamWaitEvent(cout.s, ev_out[b].e, 0));
      XCT_TRY_CUDA(cudaMemcpyAsync(yout, Yn[b], sizeof(float) * St * nout, cudaMemcpyDeviceToHost,
                                   cout.s));
      XCT_TRY_CUDA(cudaEventRecord(ev_d2h[b].e, cout.s));
    } else {
      XCT_TRY(to_natural(Yi[b], yout, out_inv, nout, St, st, 1, s));
    }
  }
  XCT_TRY_CUDA(cudaStreamSynchronize(cin.s));
  XCT_TRY_CUDA(cudaStreamSynchronize(cout.s));
  return check_kernel_flag(p, s);
}

xct_status apply_impl(Plan& p, bool transposed, const float* in, float* out, int32_t S,
                      cudaStream_t s) {
  const Layout& L = transposed ? p.lat : p.la;
  const int32_t* in_inv = transposed ? p.ray_inv : p.pix_inv;
  const int32_t* out_inv = transposed ? p.pix_inv : p.ray_inv;
  const int64_t nin = L.ncols, nout = L.nrows;
  const int st = pick_slices_per_tile(p.storage, S);
  const int ntiles = (S + st - 1) / st;
  const int S_pad = st * ntiles;
  const bool in_host = is_host_pointer(in), out_host = is_host_pointer(out);
  if ((in_host || out_host) && ntiles > 1)
    return apply_pipelined(p, transposed, in, out, S, st, ntiles, in_host, out_host, s);
  Arena ar(s);
  DevView iv, ov;
  XCT_TRY(device_view(in, (size_t)S * nin, true, ar, s, iv));
  XCT_TRY(device_view(out, (size_t)S * nout, false, ar, s, ov));
  float *Xi, *Yi;
  uint32_t* mx;
  XCT_TRY(ar.get(&Xi, (size_t)nin * S_pad));
  XCT_TRY(ar.get(&Yi, (size_t)nout * S_pad));
  XCT_TRY(ar.get(&mx, (size_t)S_pad));
  uint16_t* h16 = nullptr;
  if (stages16(p.storage)) XCT_TRY(ar.get(&h16, (size_t)nin * S_pad));
  int* work;
  XCT_TRY(ar.get(&work, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(uint32_t) * S_pad, s));
  XCT_TRY(to_internal(iv.dev, Xi, in_inv, nin, S, st, ntiles, mx, s));
  SpmmArgs a{&L, Xi, Yi, st, ntiles, p.storage, p.mat_scale_exp, mx, nullptr, h16, work, p.err};
  XCT_TRY(spmm(a, s));
  XCT_TRY(to_natural(Yi, ov.dev, out_inv, nout, S, st, ntiles, s));
  if (ov.host) {
    XCT_TRY_CUDA(cudaMemcpyAsync(out, ov.dev, sizeof(float) * S * nout, cudaMemcpyDeviceToHost, s));
    return check_kernel_flag(p, s);
  }
  return XCT_OK;
}

bool is_finite_d(double v) { return isfinite(v) != 0; }

}  // namespace
}  // namespace xct

using namespace xct;

extern "C" {

xct_status xct_plan(const xct_geometry* g, xct_dtype storage, uint32_t flags, void* stream,
                    xct_plan_t* out) {
  Trace trace_("xct_plan");
  if (!out) {
    set_error("out is NULL");
    return XCT_ERR_INVALID;
  }
  *out = nullptr;
  if (!g) {
    set_error("geometry is NULL");
    return XCT_ERR_INVALID;
  }
  if (g->n < 1 || g->n > 32768) {
    set_error("n = %d outside [1, 32768]", g->n);
    return XCT_ERR_INVALID;
  }
  if (g->n_angles < 1 || g->n_det < 1 || (int64_t)g->n_angles * g->n_det >= (1ll << 31)) {
    set_error("n_angles = %d, n_det = %d: need >= 1 each and a product < 2^31", g->n_angles,
              g->n_det);
    return XCT_ERR_INVALID;
  }
  if (g->hilbert_tile < 0 || g->hilbert_tile > 4096) {
    set_error("hilbert_tile = %d outside [0, 4096]", g->hilbert_tile);
    return XCT_ERR_INVALID;
  }
  if (!is_finite_d(g->det_spacing) || g->det_spacing == 0.0 || !is_finite_d(g->det_offset) ||
      !is_finite_d(g->min_seg) || g->min_seg < 0.0) {
    set_error("det_spacing must be finite and nonzero, det_offset finite, min_seg finite >= 0");
    return XCT_ERR_INVALID;
  }
  if (!valid_storage(storage)) {
    set_error("storage %d is not XCT_F32, XCT_F16, XCT_BF16, XCT_F16A or XCT_BF16A", (int)storage);
    return XCT_ERR_INVALID;
  }
  if (flags & ~(XCT_PLAN_KEEP_F64 | XCT_PLAN_AUTOTUNE | XCT_PLAN_FEW_SLICES | XCT_PLAN_NARROW_TILES |
                XCT_PLAN_PAIRED_ROWS)) {
    set_error("unknown plan flags 0x%x", flags);
    return XCT_ERR_INVALID;
  }
  if ((flags & XCT_PLAN_NARROW_TILES) && !matrix16(storage)) {
    set_error("XCT_PLAN_NARROW_TILES needs a 16-bit matrix storage (XCT_F16, XCT_BF16, XCT_F16A, XCT_BF16A)");
    return XCT_ERR_INVALID;
  }
  if ((flags & XCT_PLAN_FEW_SLICES) && !stages16(storage)) {
    set_error("XCT_PLAN_FEW_SLICES needs XCT_F16 or XCT_BF16 storage");
    return XCT_ERR_INVALID;
  }
  if ((flags & XCT_PLAN_PAIRED_ROWS) && !stages16(storage)) {
    set_error("XCT_PLAN_PAIRED_ROWS needs XCT_F16 or XCT_BF16 storage");
    return XCT_ERR_INVALID;
  }
  std::unique_ptr<xct_plan_s> p(new xct_plan_s());
  p->g = *g;
  p->g.cos_sin = nullptr;
  p->storage = storage;
  p->flags = flags;
  p->cs.resize((size_t)2 * g->n_angles);
  for (int k = 0; k < g->n_angles; ++k) {
    if (g->cos_sin) {
      p->cs[2 * k] = g->cos_sin[2 * k];
      p->cs[2 * k + 1] = g->cos_sin[2 * k + 1];
    } else {
      const double th = (double)k * M_PI / (double)g->n_angles;
      p->cs[2 * k] = cos(th);
      p->cs[2 * k + 1] = sin(th);
    }
    if (!is_finite_d(p->cs[2 * k]) || !is_finite_d(p->cs[2 * k + 1])) {
      set_error("angle table entry %d is not finite", k);
      return XCT_ERR_INVALID;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    set_error("no CUDA device");
    return XCT_ERR_CUDA;
  }
  xct_status st = build_plan(*p, s);
  if (st != XCT_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  // the fixed array of xct_project_noalloc is loaded with its module on first
  // use; taking its address here makes it resident on this device while the
  // caller is still allowed to allocate (a failure here is reported again,
  // and only, by xct_project_noalloc)
  noalloc_reserve(p->device);
  *out = p.release();
  return XCT_OK;
}

void xct_free(xct_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  plan->mem.stream = nullptr;
  delete plan;
}

xct_status xct_project(xct_plan_t plan, const float* x, float* y, int32_t S, void* stream) {
  Trace trace_("xct_project");
  XCT_TRY(check_plan(plan));
  if (S < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  return apply_impl(*plan, false, x, y, S, static_cast<cudaStream_t>(stream));
}

xct_status xct_backproject(xct_plan_t plan, const float* y, float* x, int32_t S, void* stream) {
  Trace trace_("xct_backproject");
  XCT_TRY(check_plan(plan));
  if (S < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  return apply_impl(*plan, true, y, x, S, static_cast<cudaStream_t>(stream));
}

xct_status xct_cgls(xct_plan_t plan, const float* y, float* x, int32_t S, int32_t iters,
                    uint32_t flags, double* resid, void* stream) {
  Trace trace_("xct_cgls");
  XCT_TRY(check_plan(plan));
  if (S < 0 || iters < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d, iters = %d)", S, iters);
    return XCT_ERR_INVALID;
  }
  if (flags & ~(XCT_CGLS_X0 | XCT_CGLS_NO_GRAPH | XCT_CGLS_TIMING)) {
    set_error("unknown CGLS flags 0x%x", flags);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  return cgls_impl(*plan, y, x, S, iters, flags, resid, nullptr, static_cast<cudaStream_t>(stream));
}

xct_status xct_project_matfree(xct_plan_t plan, const float* x, float* y, int32_t S, void* stream) {
  Trace trace_("xct_project_matfree");
  XCT_TRY(check_plan(plan));
  if (S < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(s);
  DevView xv, yv;
  XCT_TRY(device_view(x, (size_t)S * p.npix, true, ar, s, xv));
  XCT_TRY(device_view(y, (size_t)S * p.nray, false, ar, s, yv));
  double* cs_dev;
  XCT_TRY(ar.get(&cs_dev, 2 * (size_t)p.g.n_angles));
  XCT_TRY_CUDA(cudaMemcpyAsync(cs_dev, p.cs.data(), sizeof(double) * 2 * p.g.n_angles,
                               cudaMemcpyHostToDevice, s));
  XCT_TRY(matfree_project(p, cs_dev, xv.dev, yv.dev, S, s));
  if (yv.host) {
    XCT_TRY_CUDA(cudaMemcpyAsync(y, yv.dev, sizeof(float) * S * p.nray, cudaMemcpyDeviceToHost, s));
  }
  // the angle table copy comes from host memory owned by the plan: wait for it
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  return XCT_OK;
}

static xct_status apply_f64(xct_plan_t plan, bool transposed, const double* in, double* out, int32_t S,
                     void* stream) {
  XCT_TRY(check_plan(plan));
  if (S < 0 || ((!in || !out) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  Plan& p = *plan;
  if (!p.a_val) {
    set_error("the FP64 path needs a plan built with XCT_PLAN_KEEP_F64");
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nin = transposed ? p.nray : p.npix, nout = transposed ? p.npix : p.nray;
  Arena ar(s);
  DevViewT<double> iv, ov;
  XCT_TRY(device_view(in, (size_t)S * nin, true, ar, s, iv));
  XCT_TRY(device_view(out, (size_t)S * nout, false, ar, s, ov));
  XCT_TRY(f64_apply(p, transposed, iv.dev, ov.dev, S, s));
  if (ov.host) {
    XCT_TRY_CUDA(cudaMemcpyAsync(out, ov.dev, sizeof(double) * S * nout, cudaMemcpyDeviceToHost, s));
    XCT_TRY_CUDA(cudaStreamSynchronize(s));
  }
  return XCT_OK;
}

xct_status xct_project_f64(xct_plan_t plan, const double* x, double* y, int32_t S, void* stream) {
  Trace trace_("xct_project_f64");
  return apply_f64(plan, false, x, y, S, stream);
}

xct_status xct_backproject_f64(xct_plan_t plan, const double* y, double* x, int32_t S,
                               void* stream) {
  Trace trace_("xct_backproject_f64");
  return apply_f64(plan, true, y, x, S, stream);
}

xct_status xct_cgls_f64(xct_plan_t plan, const double* y, double* x, int32_t S, int32_t iters,
                        uint32_t flags, double* resid, void* stream) {
  Trace trace_("xct_cgls_f64");
  XCT_TRY(check_plan(plan));
  if (S < 0 || iters < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d, iters = %d)", S, iters);
    return XCT_ERR_INVALID;
  }
  if (flags & ~XCT_CGLS_X0) {
    set_error("unknown FP64 CGLS flags 0x%x", flags);
    return XCT_ERR_INVALID;
  }
  Plan& p = *plan;
  if (!p.a_val) {
    set_error("the FP64 path needs a plan built with XCT_PLAN_KEEP_F64");
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool x0 = (flags & XCT_CGLS_X0) != 0;
  Arena ar(s);
  DevViewT<double> yv, xv;
  XCT_TRY(device_view(y, (size_t)S * p.nray, true, ar, s, yv));
  XCT_TRY(device_view(x, (size_t)S * p.npix, x0, ar, s, xv));
  double* log = nullptr;
  if (resid) XCT_TRY(ar.get(&log, (size_t)(iters + 1) * S * 2));
  int any = 0;
  XCT_TRY(f64_cgls(p, yv.dev, xv.dev, S, iters, x0, log, &any, s));
  if (resid)
    XCT_TRY_CUDA(cudaMemcpyAsync(resid, log, sizeof(double) * (iters + 1) * S * 2,
                                 is_host_pointer(resid) ? cudaMemcpyDeviceToHost
                                                        : cudaMemcpyDeviceToDevice, s));
  if (xv.host)
    XCT_TRY_CUDA(cudaMemcpyAsync(x, xv.dev, sizeof(double) * S * p.npix, cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  if (!any) {
    set_error("CGLS breakdown: every slice has A^T r_0 = 0");
    return XCT_ERR_BREAKDOWN;
  }
  return XCT_OK;
}

xct_status xct_backproject_matfree(xct_plan_t plan, const float* y, float* x, int32_t S,
                                   void* stream) {
  Trace trace_("xct_backproject_matfree");
  XCT_TRY(check_plan(plan));
  if (S < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d)", S);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(s);
  DevView yv, xv;
  XCT_TRY(device_view(y, (size_t)S * p.nray, true, ar, s, yv));
  XCT_TRY(device_view(x, (size_t)S * p.npix, false, ar, s, xv));
  double* cs_dev;
  XCT_TRY(ar.get(&cs_dev, 2 * (size_t)p.g.n_angles));
  XCT_TRY_CUDA(cudaMemcpyAsync(cs_dev, p.cs.data(), sizeof(double) * 2 * p.g.n_angles,
                               cudaMemcpyHostToDevice, s));
  XCT_TRY(matfree_backproject(p, cs_dev, yv.dev, xv.dev, S, s));
  if (xv.host) {
    XCT_TRY_CUDA(cudaMemcpyAsync(x, xv.dev, sizeof(float) * S * p.npix, cudaMemcpyDeviceToHost, s));
  }
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  return XCT_OK;
}

xct_status xct_cgls_matfree(xct_plan_t plan, const float* y, float* x, int32_t S, int32_t iters,
                            uint32_t flags, double* resid, void* stream) {
  Trace trace_("xct_cgls_matfree");
  XCT_TRY(check_plan(plan));
  if (S < 0 || iters < 0 || ((!x || !y) && S > 0)) {
    set_error("bad arguments (S = %d, iters = %d)", S, iters);
    return XCT_ERR_INVALID;
  }
  if (flags & ~XCT_CGLS_X0) {
    set_error("unknown matrix-free CGLS flags 0x%x", flags);
    return XCT_ERR_INVALID;
  }
  if (S == 0) return XCT_OK;
  Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool x0 = (flags & XCT_CGLS_X0) != 0;
  const int64_t npix = p.npix, nray = p.nray;
  Arena ar(s);
  DevView yv, xv;
  XCT_TRY(device_view(y, (size_t)S * nray, true, ar, s, yv));
  XCT_TRY(device_view(x, (size_t)S * npix, x0, ar, s, xv));
  double* cs_dev;
  XCT_TRY(ar.get(&cs_dev, 2 * (size_t)p.g.n_angles));
  XCT_TRY_CUDA(cudaMemcpyAsync(cs_dev, p.cs.data(), sizeof(double) * 2 * p.g.n_angles,
                               cudaMemcpyHostToDevice, s));
  // natural layouts are the vector kernels' layout with one slice per tile
  float *X, *P, *Sv, *R, *Q;
  double *dpart, *gpart, *rpart, *log;
  CglsScalars sc{};
  XCT_TRY(ar.get(&X, (size_t)npix * S));
  XCT_TRY(ar.get(&P, (size_t)npix * S));
  XCT_TRY(ar.get(&Sv, (size_t)npix * S));
  XCT_TRY(ar.get(&R, (size_t)nray * S));
  XCT_TRY(ar.get(&Q, (size_t)nray * S));
  XCT_TRY(ar.get(&dpart, (size_t)S * kVecBlocks));
  XCT_TRY(ar.get(&gpart, (size_t)S * kVecBlocks));
  XCT_TRY(ar.get(&rpart, (size_t)S * kVecBlocks));
  XCT_TRY(ar.get(&log, (size_t)(iters + 1) * S * 2));
  XCT_TRY(ar.get(&sc.gamma, (size_t)S));
  XCT_TRY(ar.get(&sc.alpha, (size_t)S));
  XCT_TRY(ar.get(&sc.beta, (size_t)S));
  XCT_TRY(ar.get(&sc.active, (size_t)S));
  XCT_TRY(ar.get(&sc.active0, (size_t)S));
  XCT_TRY(ar.get(&sc.max_r, (size_t)S));
  XCT_TRY(ar.get(&sc.max_p, (size_t)S));
  // the recurrence of xct_cgls (Table IV footnote: one initial back
  // projection, then one projection and one back projection per iteration)
  XCT_TRY_CUDA(cudaMemcpyAsync(R, yv.dev, sizeof(float) * nray * S, cudaMemcpyDeviceToDevice, s));
  if (x0) {
    XCT_TRY_CUDA(cudaMemcpyAsync(X, xv.dev, sizeof(float) * npix * S, cudaMemcpyDeviceToDevice, s));
    XCT_TRY(matfree_project(p, cs_dev, X, Q, S, s));
    XCT_TRY(cgls_residual(R, Q, nray, 1, S, sc.max_r, rpart, s));
  } else {
    XCT_TRY_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * npix * S, s));
    XCT_TRY(cgls_residual(R, nullptr, nray, 1, S, sc.max_r, rpart, s));
  }
  XCT_TRY(matfree_backproject(p, cs_dev, R, Sv, S, s));
  XCT_TRY(cgls_residual(Sv, nullptr, npix, 1, S, sc.max_p, gpart, s));
  XCT_TRY(cgls_init_scalars(gpart, kVecBlocks, rpart, sc, log, S, s));
  XCT_TRY_CUDA(cudaMemsetAsync(P, 0, sizeof(float) * npix * S, s));
  XCT_TRY(cgls_update_p(P, Sv, npix, 1, S, sc, s));
  for (int it = 1; it <= iters; ++it) {
    XCT_TRY(matfree_project(p, cs_dev, P, Q, S, s));
    XCT_TRY(cgls_residual(Q, nullptr, nray, 1, S, sc.max_r, dpart, s));
    XCT_TRY(cgls_alpha(dpart, kVecBlocks, sc, S, s));
    XCT_TRY(cgls_update_xr(X, P, npix, R, Q, nray, 1, S, sc, rpart, s));
    XCT_TRY(matfree_backproject(p, cs_dev, R, Sv, S, s));
    XCT_TRY(cgls_residual(Sv, nullptr, npix, 1, S, sc.max_p, gpart, s));
    XCT_TRY(cgls_beta(gpart, kVecBlocks, rpart, sc, log + (size_t)it * S * 2, S, s));
    XCT_TRY(cgls_update_p(P, Sv, npix, 1, S, sc, s));
  }
  XCT_TRY_CUDA(cudaMemcpyAsync(xv.dev, X, sizeof(float) * npix * S, cudaMemcpyDeviceToDevice, s));
  if (xv.host)
    XCT_TRY_CUDA(cudaMemcpyAsync(x, xv.dev, sizeof(float) * S * npix, cudaMemcpyDeviceToHost, s));
  if (resid)
    XCT_TRY_CUDA(cudaMemcpyAsync(resid, log, sizeof(double) * (iters + 1) * S * 2,
                                 is_host_pointer(resid) ? cudaMemcpyDeviceToHost
                                                        : cudaMemcpyDeviceToDevice, s));
  std::vector<int> act0((size_t)S);
  XCT_TRY_CUDA(cudaMemcpyAsync(act0.data(), sc.active0, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  bool any = false;
  for (int i = 0; i < S; ++i) any = any || act0[i];
  if (!any) {
    set_error("CGLS breakdown: every slice has A^T r_0 = 0");
    return XCT_ERR_BREAKDOWN;
  }
  return XCT_OK;
}

int64_t xct_cgls_state_bytes(xct_plan_t plan, int32_t S) {
  if (!plan || S < 1) return 0;
  return (int64_t)state_bytes(plan->npix, plan->nray, S);
}

xct_status xct_cgls_state(xct_plan_t plan, const float* y, float* x, int32_t S, int32_t iters,
                          uint32_t flags, double* resid, void* state, void* stream) {
  Trace trace_("xct_cgls_state");
  XCT_TRY(check_plan(plan));
  const uint32_t known = XCT_CGLS_X0 | XCT_CGLS_NO_GRAPH | XCT_CGLS_TIMING | XCT_CGLS_SAVE |
                         XCT_CGLS_RESUME;
  if (S < 1 || iters < 0 || !x || !state || (!y && !(flags & XCT_CGLS_RESUME)) || (flags & ~known) ||
      !(flags & (XCT_CGLS_SAVE | XCT_CGLS_RESUME))) {
    set_error("bad arguments (S = %d, iters = %d, flags 0x%x; SAVE or RESUME needed)", S, iters,
              flags);
    return XCT_ERR_INVALID;
  }
  return cgls_impl(*plan, y, x, S, iters, flags, resid, state, static_cast<cudaStream_t>(stream));
}

xct_status xct_plan_stats(xct_plan_t plan, xct_stats* out) {
  XCT_TRY(check_plan(plan));
  if (!out) {
    set_error("out is NULL");
    return XCT_ERR_INVALID;
  }
  *out = plan->stats;
  return XCT_OK;
}

xct_status xct_plan_export(xct_plan_t plan, int32_t what, int64_t* rowptr, int32_t* col,
                           double* val, int64_t* nnz) {
  XCT_TRY(check_plan(plan));
  if (!nnz || what < 0 || what > 5 || (rowptr && (!col || !val))) {
    set_error("bad export arguments");
    return XCT_ERR_INVALID;
  }
  XCT_TRY_CUDA(cudaDeviceSynchronize());
  return export_matrix(*plan, what, rowptr, col, val, nnz);
}

xct_status xct_plan_order(xct_plan_t plan, int32_t* pix, int32_t* ray) {
  XCT_TRY(check_plan(plan));
  XCT_TRY_CUDA(cudaDeviceSynchronize());
  if (pix)
    XCT_TRY_CUDA(cudaMemcpy(pix, plan->pix_order, sizeof(int32_t) * plan->npix,
                            cudaMemcpyDeviceToHost));
  if (ray)
    XCT_TRY_CUDA(cudaMemcpy(ray, plan->ray_order, sizeof(int32_t) * plan->nray,
                            cudaMemcpyDeviceToHost));
  return XCT_OK;
}

xct_status xct_set_allocator(xct_alloc_fn alloc, xct_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) {
    set_error("set both allocator callbacks or neither");
    return XCT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_hook_mu);
  g_hook.alloc = alloc;
  g_hook.release = release;
  g_hook.ctx = ctx;
  return XCT_OK;
}

const char* xct_last_error(void) { return g_err; }

int64_t xct_launch_count(void) { return g_launches.load(); }

xct_status xct_set_wait_limit(uint64_t ns, uint64_t* previous) {
  if (ns > 60000000000ull) {
    set_error("wait limit %llu ns above 60 s", (unsigned long long)ns);
    return XCT_ERR_INVALID;
  }
  const uint64_t old = g_wait_ns.exchange(ns);
  if (previous) *previous = old;
  return XCT_OK;
}

xct_status xct_plan_check(xct_plan_t plan, void* stream) {
  if (!plan) {
    set_error("plan is NULL");
    return XCT_ERR_INVALID;
  }
  Plan& p = *static_cast<Plan*>(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int e = 0;
  XCT_TRY_CUDA(cudaMemcpyAsync(&e, p.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  XCT_TRY_CUDA(cudaStreamSynchronize(s));
  if (e) {
    XCT_TRY_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), s));
    XCT_TRY_CUDA(cudaStreamSynchronize(s));
    set_error("a bounded wait in a product kernel of this plan ran out; its results are invalid");
    return XCT_ERR_TIMEOUT;
  }
  return XCT_OK;
}

const char* xct_version(void) { return "xct 0.1.0 (sm_103a)"; }

}  // extern "C"

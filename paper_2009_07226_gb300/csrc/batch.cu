// xct_cgls_batch: many CGLS jobs of uneven geometry and slice count in one
// go (batch processing of slices sharing A, Sec. II-B / III-A2, extended to
// several geometries).
//
//  * jobs are grouped by plan (one memoized matrix per geometry) and the
//    slices of a group are concatenated: slices are independent problems
//    with their own CGLS scalars, so a group is one batched solve;
//  * each group's slice-tile width is chosen by timing the candidate widths
//    on the group's plan (XCT_BATCH_AUTOTUNE; cached in the plan) or by the
//    default rule;
//  * every product phase of all groups that share a kernel configuration is
//    one persistent launch over their combined work list; the vector and
//    scalar kernels run per group;
//  * the whole batch is one CUDA graph.
#include <algorithm>
#include <map>
#include <vector>

#include "xct_internal.cuh"
#include "xct_vec.cuh"

namespace xct {
namespace {

bool dev_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct Group {
  Plan* p = nullptr;
  std::vector<int> jobs;       // indices into the job list
  std::vector<int> off;        // slice offset of each job in the group
  int S = 0, st = 1, ntiles = 0, S_pad = 0;
  float *Y = nullptr, *Xn = nullptr;                  // natural concatenated y, x
  float *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr, *Sv = nullptr;
  uint16_t *h_pix = nullptr, *h_ray = nullptr;
  double *dpart = nullptr, *gpart = nullptr, *rpart = nullptr, *log = nullptr;
  uint32_t* max_x = nullptr;
  CglsScalars sc{};
  SpmmArgs fwd() const {
    return SpmmArgs{&p->la, P, Q, st, ntiles, p->storage, p->mat_scale_exp, sc.max_p, dpart,
                    h_pix, nullptr, p->err};
  }
  SpmmArgs bwd() const {
    return SpmmArgs{&p->lat, R, Sv, st, ntiles, p->storage, p->mat_scale_exp, sc.max_r, gpart,
                    h_ray, nullptr, p->err};
  }
};

// Slice-tile width for S slices on plan p: measured (cached in the plan) or
// the default rule.
xct_status choose_tile(Plan& p, int S, bool tune, cudaStream_t s, int* out) {
  if (!tune) {
    *out = pick_slices_per_tile(p.storage, S);
    return XCT_OK;
  }
  auto it = p.tile_choice.find(S);
  if (it != p.tile_choice.end()) {
    *out = it->second;
    return XCT_OK;
  }
  const std::vector<int> cand = stages16(p.storage) ? std::vector<int>{8, 16, 32, 64}
                                                     : (matrix16(p.storage) ? std::vector<int>{8, 16, 32}
                                                                            : std::vector<int>{4, 8, 16, 32});
  double best = 1e300;
  int best_st = pick_slices_per_tile(p.storage, S);
  for (int st : cand) {
    const int ntiles = (S + st - 1) / st;
    const int S_pad = ntiles * st;
    Arena ar(s);
    float *xi, *yi;
    uint16_t* h = nullptr;
    uint32_t* mx;
    int* work;
    XCT_TRY(ar.get(&xi, (size_t)p.npix * S_pad));
    XCT_TRY(ar.get(&yi, (size_t)p.nray * S_pad));
    if (stages16(p.storage)) XCT_TRY(ar.get(&h, (size_t)std::max(p.npix, p.nray) * S_pad));
    XCT_TRY(ar.get(&mx, (size_t)S_pad));
    XCT_TRY(ar.get(&work, 1));
    XCT_TRY_CUDA(cudaMemsetAsync(xi, 0, sizeof(float) * p.npix * S_pad, s));
    XCT_TRY_CUDA(cudaMemsetAsync(yi, 0, sizeof(float) * p.nray * S_pad, s));
    XCT_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(uint32_t) * S_pad, s));
    SpmmArgs f{&p.la, xi, yi, st, ntiles, p.storage, p.mat_scale_exp, mx, nullptr, h, work, p.err};
    SpmmArgs b{&p.lat, yi, xi, st, ntiles, p.storage, p.mat_scale_exp, mx, nullptr, h, work, p.err};
    cudaEvent_t e0, e1;
    XCT_TRY_CUDA(cudaEventCreate(&e0));
    XCT_TRY_CUDA(cudaEventCreate(&e1));
    xct_status st_run = spmm(f, s);  // warm-up
    if (st_run == XCT_OK) st_run = spmm(b, s);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && st_run == XCT_OK; ++r) {
      st_run = spmm(f, s);
      if (st_run == XCT_OK) st_run = spmm(b, s);
    }
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    XCT_TRY(st_run);
    if (e != cudaSuccess) {
      set_error("autotune timing failed: %s", cudaGetErrorString(e));
      return XCT_ERR_CUDA;
    }
    if (ms < best) {
      best = ms;
      best_st = st;
    }
  }
  p.tile_choice[S] = best_st;
  *out = best_st;
  return XCT_OK;
}

xct_status alloc_group(Group& g, int iters, Arena& ar) {
  Plan& p = *g.p;
  const size_t np = (size_t)p.npix * g.S_pad, nr = (size_t)p.nray * g.S_pad;
  XCT_TRY(ar.get(&g.Y, (size_t)g.S * p.nray));
  XCT_TRY(ar.get(&g.Xn, (size_t)g.S * p.npix));
  XCT_TRY(ar.get(&g.X, np));
  XCT_TRY(ar.get(&g.P, np));
  XCT_TRY(ar.get(&g.Sv, np));
  XCT_TRY(ar.get(&g.R, nr));
  XCT_TRY(ar.get(&g.Q, nr));
  if (stages16(p.storage)) {
    XCT_TRY(ar.get(&g.h_pix, np));
    XCT_TRY(ar.get(&g.h_ray, nr));
  }
  XCT_TRY(ar.get(&g.dpart, (size_t)g.S_pad * std::max(p.la.nblocks, 1)));
  XCT_TRY(ar.get(&g.gpart, (size_t)g.S_pad * std::max(p.lat.nblocks, 1)));
  XCT_TRY(ar.get(&g.rpart, (size_t)g.S_pad * kVecBlocks));
  XCT_TRY(ar.get(&g.log, (size_t)(iters + 1) * g.S_pad * 2));
  XCT_TRY(ar.get(&g.max_x, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.gamma, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.alpha, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.beta, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.active, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.active0, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.max_r, (size_t)g.S_pad));
  XCT_TRY(ar.get(&g.sc.max_p, (size_t)g.S_pad));
  return XCT_OK;
}

// One product phase for all groups: the 16-bit staging copies per group,
// then one persistent launch per run of groups sharing a kernel
// configuration (or per-group launches where the persistent form does not
// apply).
xct_status product_phase(std::vector<Group>& G, bool forward, int* work, cudaStream_t s) {
  std::vector<SpmmArgs> all;
  for (auto& g : G) {
    SpmmArgs a = forward ? g.fwd() : g.bwd();
    a.work = work;
    XCT_TRY(spmm_stage(a, s));
    all.push_back(a);
  }
  size_t i = 0;
  while (i < all.size()) {
    size_t j = i + 1;
    while (j < all.size() && (int)(j - i) < kMaxPipeProducts && all[j].storage == all[i].storage &&
           all[j].st == all[i].st &&
           spmm_pipe_multi_applies(&all[i], (int)(j - i + 1)))
      ++j;
    if (j - i > 1 || spmm_pipe_multi_applies(&all[i], 1))
      XCT_TRY(spmm_pipe_multi(&all[i], (int)(j - i), s));
    else
      XCT_TRY(spmm_run(all[i], s));
    i = j;
  }
  return XCT_OK;
}

xct_status enqueue_batch(std::vector<Group>& G, const xct_job* jobs, int iters, bool x0, int* work,
                         cudaStream_t s) {
  for (auto& g : G) {
    Plan& p = *g.p;
    for (size_t k = 0; k < g.jobs.size(); ++k) {
      const xct_job& jb = jobs[g.jobs[k]];
      XCT_TRY_CUDA(cudaMemcpyAsync(g.Y + (size_t)g.off[k] * p.nray, jb.y,
                                   sizeof(float) * jb.S * p.nray, cudaMemcpyDeviceToDevice, s));
      if (x0)
        XCT_TRY_CUDA(cudaMemcpyAsync(g.Xn + (size_t)g.off[k] * p.npix, jb.x,
                                     sizeof(float) * jb.S * p.npix, cudaMemcpyDeviceToDevice, s));
    }
    XCT_TRY_CUDA(cudaMemsetAsync(g.sc.max_r, 0, sizeof(uint32_t) * g.S_pad, s));
    XCT_TRY(to_internal(g.Y, g.R, p.ray_inv, p.nray, g.S, g.st, g.ntiles, g.sc.max_r, s));
    if (x0) {
      XCT_TRY_CUDA(cudaMemsetAsync(g.max_x, 0, sizeof(uint32_t) * g.S_pad, s));
      XCT_TRY(to_internal(g.Xn, g.X, p.pix_inv, p.npix, g.S, g.st, g.ntiles, g.max_x, s));
      SpmmArgs a{&p.la, g.X, g.Q, g.st, g.ntiles, p.storage, p.mat_scale_exp, g.max_x, nullptr,
                 g.h_pix, work, p.err};
      XCT_TRY(spmm(a, s));
      XCT_TRY_CUDA(cudaMemsetAsync(g.sc.max_r, 0, sizeof(uint32_t) * g.S_pad, s));
      XCT_TRY(cgls_residual(g.R, g.Q, p.nray, g.st, g.ntiles, g.sc.max_r, g.rpart, s));
    } else {
      XCT_TRY_CUDA(cudaMemsetAsync(g.X, 0, sizeof(float) * p.npix * g.S_pad, s));
      XCT_TRY(cgls_residual(g.R, nullptr, p.nray, g.st, g.ntiles, g.sc.max_r, g.rpart, s));
    }
    XCT_TRY_CUDA(cudaMemsetAsync(g.P, 0, sizeof(float) * p.npix * g.S_pad, s));
  }
  XCT_TRY(product_phase(G, false, work, s));
  for (auto& g : G) {
    XCT_TRY(cgls_init_scalars(g.gpart, spmm_dot_count(g.bwd()), g.rpart, g.sc, g.log, g.S_pad, s));
    XCT_TRY(cgls_update_p(g.P, g.Sv, g.p->npix, g.st, g.ntiles, g.sc, s));
  }
  for (int it = 1; it <= iters; ++it) {
    XCT_TRY(product_phase(G, true, work, s));
    for (auto& g : G) {
      XCT_TRY(cgls_alpha(g.dpart, spmm_dot_count(g.fwd()), g.sc, g.S_pad, s));
      XCT_TRY(cgls_update_xr(g.X, g.P, g.p->npix, g.R, g.Q, g.p->nray, g.st, g.ntiles, g.sc,
                             g.rpart, s));
    }
    XCT_TRY(product_phase(G, false, work, s));
    for (auto& g : G) {
      XCT_TRY(cgls_beta(g.gpart, spmm_dot_count(g.bwd()), g.rpart, g.sc,
                        g.log + (size_t)it * g.S_pad * 2, g.S_pad, s));
      XCT_TRY(cgls_update_p(g.P, g.Sv, g.p->npix, g.st, g.ntiles, g.sc, s));
    }
  }
  for (auto& g : G) {
    Plan& p = *g.p;
    XCT_TRY(to_natural(g.X, g.Xn, p.pix_inv, p.npix, g.S, g.st, g.ntiles, s));
    for (size_t k = 0; k < g.jobs.size(); ++k) {
      const xct_job& jb = jobs[g.jobs[k]];
      XCT_TRY_CUDA(cudaMemcpyAsync(jb.x, g.Xn + (size_t)g.off[k] * p.npix,
                                   sizeof(float) * jb.S * p.npix, cudaMemcpyDeviceToDevice, s));
    }
  }
  return XCT_OK;
}

}  // namespace
}  // namespace xct

using namespace xct;

extern "C" xct_status xct_cgls_batch(const xct_job* jobs, int32_t n_jobs, int32_t iters,
                                     uint32_t flags, void* stream) {
  if (n_jobs < 0 || iters < 0 || (n_jobs > 0 && !jobs) ||
      (flags & ~(XCT_CGLS_X0 | XCT_CGLS_NO_GRAPH | XCT_BATCH_AUTOTUNE))) {
    set_error("xct_cgls_batch: bad arguments");
    return XCT_ERR_INVALID;
  }
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  std::vector<Group> G;
  std::map<Plan*, int> gi;
  for (int j = 0; j < n_jobs; ++j) {
    const xct_job& jb = jobs[j];
    if (!jb.plan || jb.S < 0 || (jb.S > 0 && (!jb.y || !jb.x))) {
      set_error("xct_cgls_batch: job %d is invalid", j);
      return XCT_ERR_INVALID;
    }
    if (jb.S == 0) continue;
    if (!dev_accessible(jb.y) || !dev_accessible(jb.x) || (jb.resid && !dev_accessible(jb.resid))) {
      set_error("xct_cgls_batch: job %d: buffers must be device memory", j);
      return XCT_ERR_INVALID;
    }
    Plan* p = static_cast<Plan*>(jb.plan);
    auto f = gi.find(p);
    if (f == gi.end()) {
      gi[p] = (int)G.size();
      G.emplace_back();
      G.back().p = p;
      f = gi.find(p);
    }
    Group& g = G[f->second];
    g.jobs.push_back(j);
    g.off.push_back(g.S);
    g.S += jb.S;
  }
  if (G.empty()) return XCT_OK;
  const bool tune = (flags & XCT_BATCH_AUTOTUNE) != 0;
  for (auto& g : G) {
    XCT_TRY(choose_tile(*g.p, g.S, tune, us, &g.st));
    g.ntiles = (g.S + g.st - 1) / g.st;
    g.S_pad = g.ntiles * g.st;
  }
  Arena ar(us);
  for (auto& g : G) XCT_TRY(alloc_group(g, iters, ar));
  int* work;
  XCT_TRY(ar.get(&work, 1));
  const bool x0 = (flags & XCT_CGLS_X0) != 0;
  if (flags & XCT_CGLS_NO_GRAPH) {
    XCT_TRY(enqueue_batch(G, jobs, iters, x0, work, us));
  } else {
    cudaStream_t cs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (cs) cudaStreamDestroy(cs);
    };
    xct_status st = XCT_OK;
    cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, us);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, e0, 0);
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      st = enqueue_batch(G, jobs, iters, x0, work, cs);
      cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      if (st == XCT_OK && ee != cudaSuccess) ce = ee;
    }
    if (st == XCT_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (st == XCT_OK && ce == cudaSuccess) ce = cudaGraphLaunch(exec, cs);
    if (st == XCT_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, cs);
    if (st == XCT_OK && ce == cudaSuccess) ce = cudaStreamWaitEvent(us, e1, 0);
    if (st == XCT_OK && ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    cleanup();
    if (st != XCT_OK) return st;
    if (ce != cudaSuccess) {
      set_error("xct_cgls_batch graph: %s", cudaGetErrorString(ce));
      return XCT_ERR_CUDA;
    }
  }
  // per-job residual logs: the job's slices of the group log
  for (auto& g : G)
    for (size_t k = 0; k < g.jobs.size(); ++k) {
      const xct_job& jb = jobs[g.jobs[k]];
      if (!jb.resid) continue;
      XCT_TRY_CUDA(cudaMemcpy2DAsync(jb.resid, sizeof(double) * 2 * jb.S,
                                     g.log + (size_t)g.off[k] * 2, sizeof(double) * 2 * g.S_pad,
                                     sizeof(double) * 2 * jb.S, iters + 1, cudaMemcpyDeviceToDevice,
                                     us));
    }
  int kerr = 0;
  for (auto& g : G) {
    int e = 0;
    XCT_TRY_CUDA(cudaMemcpyAsync(&e, g.p->err, sizeof(int), cudaMemcpyDeviceToHost, us));
    XCT_TRY_CUDA(cudaStreamSynchronize(us));
    if (e) {
      kerr = 1;
      XCT_TRY_CUDA(cudaMemsetAsync(g.p->err, 0, sizeof(int), us));
    }
  }
  XCT_TRY_CUDA(cudaStreamSynchronize(us));
  if (kerr) {
    set_error("a bounded wait in the product kernel ran out; results are invalid");
    return XCT_ERR_TIMEOUT;
  }
  return XCT_OK;
}

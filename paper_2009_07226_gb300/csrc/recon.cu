// xct_tv_reconstruct: the regularised reconstruction of Eq. 1 with
// R(x) = lam * TV_eps(x), minimised by Adam.  Each step runs, on the GPU:
// projection q = A x, residual r = q - y with 0.5 ||r||^2, gradient
// g = A^T r (the back projection), g += lam * grad TV_eps(x) with its value,
// the loss, and the Adam update of x.
#include "xct_internal.cuh"
#include "xct_vec.cuh"

namespace xct {
namespace {

bool on_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace xct

using namespace xct;

extern "C" xct_status xct_tv_reconstruct(xct_plan_t plan, const float* y, float* x, int32_t S,
                                         int32_t steps, double lr, double lam, double eps,
                                         uint32_t flags, double* loss, void* stream) {
  if (!plan || S < 0 || steps < 0 || ((!x || !y) && S > 0) || !(lr >= 0.0) || !(lam >= 0.0) ||
      !(eps > 0.0) || (flags & ~1u)) {
    set_error("xct_tv_reconstruct: bad arguments");
    return XCT_ERR_INVALID;
  }
  if (S == 0 || steps == 0) return XCT_OK;
  Plan& p = *static_cast<Plan*>(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = p.g.n;
  const int64_t npix = p.npix, nray = p.nray;
  const int st = pick_slices_per_tile(p.storage, S);
  const int ntiles = (S + st - 1) / st;
  const int S_pad = st * ntiles;
  const int k = p.mat_scale_exp;
  Arena ar(s);
  // caller buffers (device views; host ones are staged)
  float *yd = const_cast<float*>(y), *xd = x;
  const bool yh = on_host(y), xh = on_host(x);
  if (yh) {
    XCT_TRY(ar.get(&yd, (size_t)S * nray));
    XCT_TRY_CUDA(cudaMemcpyAsync(yd, y, sizeof(float) * S * nray, cudaMemcpyHostToDevice, s));
  }
  if (xh) {
    XCT_TRY(ar.get(&xd, (size_t)S * npix));
    if (flags & 1u)
      XCT_TRY_CUDA(cudaMemcpyAsync(xd, x, sizeof(float) * S * npix, cudaMemcpyHostToDevice, s));
  }
  float *m, *v, *g, *Xi, *Q, *R, *Yi, *Gi;
  uint16_t *h_pix = nullptr, *h_ray = nullptr;
  uint32_t *max_x, *max_r;
  double *rpart, *tvpart, *tvval, *lossd;
  int* work;
  XCT_TRY(ar.get(&m, (size_t)S * npix));
  XCT_TRY(ar.get(&v, (size_t)S * npix));
  XCT_TRY(ar.get(&g, (size_t)S * npix));
  XCT_TRY(ar.get(&Xi, (size_t)S_pad * npix));
  XCT_TRY(ar.get(&Gi, (size_t)S_pad * npix));
  XCT_TRY(ar.get(&Q, (size_t)S_pad * nray));
  XCT_TRY(ar.get(&R, (size_t)S_pad * nray));
  XCT_TRY(ar.get(&Yi, (size_t)S_pad * nray));
  if (stages16(p.storage)) {
    XCT_TRY(ar.get(&h_pix, (size_t)S_pad * npix));
    XCT_TRY(ar.get(&h_ray, (size_t)S_pad * nray));
  }
  XCT_TRY(ar.get(&max_x, (size_t)S_pad));
  XCT_TRY(ar.get(&max_r, (size_t)S_pad));
  XCT_TRY(ar.get(&rpart, (size_t)S_pad * kVecBlocks));
  XCT_TRY(ar.get(&tvpart, (size_t)S * tv_partials(n)));
  XCT_TRY(ar.get(&tvval, (size_t)S));
  XCT_TRY(ar.get(&lossd, (size_t)steps));
  XCT_TRY(ar.get(&work, 1));

  XCT_TRY(to_internal(yd, Yi, p.ray_inv, nray, S, st, ntiles, nullptr, s));
  if (!(flags & 1u)) XCT_TRY_CUDA(cudaMemsetAsync(xd, 0, sizeof(float) * S * npix, s));
  XCT_TRY_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * S * npix, s));
  XCT_TRY_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * S * npix, s));
  for (int t = 1; t <= steps; ++t) {
    XCT_TRY_CUDA(cudaMemsetAsync(max_x, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(to_internal(xd, Xi, p.pix_inv, npix, S, st, ntiles, max_x, s));
    SpmmArgs fa{&p.la, Xi, Q, st, ntiles, p.storage, k, max_x, nullptr, h_pix, work, p.err};
    XCT_TRY(spmm(fa, s));
    XCT_TRY_CUDA(cudaMemsetAsync(max_r, 0, sizeof(uint32_t) * S_pad, s));
    XCT_TRY(vec_sub_sumsq(Q, Yi, R, nray, st, ntiles, max_r, rpart, s));
    SpmmArgs ba{&p.lat, R, Gi, st, ntiles, p.storage, k, max_r, nullptr, h_ray, work, p.err};
    XCT_TRY(spmm(ba, s));
    XCT_TRY(to_natural(Gi, g, p.pix_inv, npix, S, st, ntiles, s));
    XCT_TRY(tv_launch(xd, n, S, eps, lam, g, true, tvpart, tvval, s));
    XCT_TRY(vec_loss(rpart, tvval, S, lossd + (t - 1), s));
    XCT_TRY(adam_launch(xd, g, m, v, (int64_t)S * npix, lr, 0.9, 0.999, 1e-8, t, s));
  }
  if (loss) {
    const bool lh = on_host(loss);
    XCT_TRY_CUDA(cudaMemcpyAsync(loss, lossd, sizeof(double) * steps,
                                 lh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  }
  if (xh) XCT_TRY_CUDA(cudaMemcpyAsync(x, xd, sizeof(float) * S * npix, cudaMemcpyDeviceToHost, s));
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

extern "C" xct_status xct_datafit(const float* q, const float* y, float* r, int64_t len,
                                  int32_t S, double* value, void* stream) {
  Trace trace_("xct_datafit");
  if (S < 0 || len < 0 || ((!q || !y || !r) && (int64_t)S * len > 0)) {
    set_error("xct_datafit: bad arguments (S = %d, len = %lld)", S, (long long)len);
    return XCT_ERR_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vh = value && on_host(value);
  if ((int64_t)S * len == 0) {
    if (value) {
      if (vh) *value = 0.0;
      else XCT_TRY_CUDA(cudaMemsetAsync(value, 0, sizeof(double), s));
    }
    return XCT_OK;
  }
  if (on_host(q) || on_host(y) || on_host(r)) {
    set_error("xct_datafit takes device vectors");
    return XCT_ERR_INVALID;
  }
  Arena ar(s);
  double *rpart, *zero, *val;
  XCT_TRY(ar.get(&rpart, (size_t)S * kVecBlocks));
  XCT_TRY(ar.get(&zero, (size_t)S));
  XCT_TRY(ar.get(&val, 1));
  XCT_TRY_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * S, s));
  // one slice per tile: r = q - y and the per-slice partials of ||r||^2,
  // then sum_s 0.5 ||r_s||^2 in a fixed order
  XCT_TRY(vec_sub_sumsq(q, y, r, len, 1, S, nullptr, rpart, s));
  XCT_TRY(vec_loss(rpart, zero, S, value && !vh ? value : val, s));
  if (vh) {
    XCT_TRY_CUDA(cudaMemcpyAsync(value, val, sizeof(double), cudaMemcpyDeviceToHost, s));
    XCT_TRY_CUDA(cudaStreamSynchronize(s));
  }
  return XCT_OK;
}

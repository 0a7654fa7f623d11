// CGLS vector kernels and scalars (vec.cu), used by the solver driver.
#pragma once

#include "xct_internal.cuh"

namespace xct {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 1024;  // blocks per slice tile of the vector kernels

// Per-slice CGLS state on the device (FP64 scalars), [S_pad] each.
struct CglsScalars {
  double* gamma;
  double* alpha;
  double* beta;
  int* active;
  int* active0;      // active after the initial back projection
  uint32_t* max_r;   // max |r| bits (normalisation of the back projection input)
  uint32_t* max_p;   // max |p| bits (normalisation of the projection input)
};

xct_status cgls_update_xr(float* x, const float* p, int64_t npix, float* r, const float* q,
                          int64_t nray, int st, int ntiles, const CglsScalars& sc, double* rpart,
                          cudaStream_t s);
xct_status cgls_update_p(float* p, const float* sv, int64_t npix, int st, int ntiles,
                         const CglsScalars& sc, cudaStream_t s);
xct_status cgls_residual(float* r, const float* q, int64_t nray, int st, int ntiles,
                         uint32_t* max_r, double* rpart, cudaStream_t s);
// r = q - y on the internal layout, with max |r| and ||r||^2 partials
// ([S_pad][kVecBlocks]); and the loss sum_s 0.5 ||r_s||^2 + tv[s] (s < S)
xct_status vec_sub_sumsq(const float* q, const float* y, float* r, int64_t rows, int st,
                         int ntiles, uint32_t* max_r, double* rpart, cudaStream_t s);
xct_status vec_loss(const double* rpart, const double* tv, int S, double* out, cudaStream_t s);
// Header of a saved CGLS state (xct_cgls_state); followed by gamma[S]
// (double), active[S] (int32, padded to 8 bytes), x[S][npix], r[S][nray],
// p[S][npix] (float32, natural layouts).
struct CglsStateHeader {
  uint64_t magic;
  int32_t S;
  int32_t iters_done;
  int64_t npix, nray;
};
constexpr uint64_t kCglsStateMagic = 0x31657461'74736778ull;  // "xgstate1"

xct_status cgls_restore(const double* gamma_in, const int32_t* active_in, int S,
                        const double* rpart, const CglsScalars& sc, double* log, int S_pad,
                        cudaStream_t s);
xct_status cgls_save(const CglsScalars& sc, int S, const CglsStateHeader& hdr,
                     CglsStateHeader* hdr_out, double* gamma_out, int32_t* active_out,
                     cudaStream_t s);
xct_status cgls_init_scalars(const double* gpart, int nbg, const double* rpart,
                             const CglsScalars& sc, double* log, int S_pad, cudaStream_t s);
xct_status cgls_alpha(const double* dpart, int nbd, const CglsScalars& sc, int S_pad,
                      cudaStream_t s);
xct_status cgls_beta(const double* gpart, int nbg, const double* rpart, const CglsScalars& sc,
                     double* log_k, int S_pad, cudaStream_t s);

}  // namespace xct

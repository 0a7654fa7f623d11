// The fused projection / back-projection product Y = M X for a batch of
// slices sharing the sparse matrix M (A or A^T) -- paper Sec. III-B.
//
// Design on sm_103a (what differs from Listing 1, written for V100):
//   * input buffering (Sec. III-B1, III-B4): a block owns 64 consecutive rows
//     in Hilbert order; their footprint (the distinct input rows they touch)
//     is split into stages of `cap` vectors that are gathered into shared
//     memory once per stage and reused by every row of the block;
//   * register reuse (Sec. III-B2) is taken over slices: the lanes of a group
//     hold different slices of the same row, so one packed entry feeds
//     ST FMAs and every shared-memory wavefront reads one contiguous 128-byte
//     staged vector (no bank conflicts), instead of one thread per row doing
//     random 16-byte gathers;
//   * output buffering (Sec. III-B3): per-lane FP32 accumulators, written
//     once, with the per-slice squared norm reduced in the epilogue (the CGLS
//     dot product, FP64);
//   * packing (Sec. III-C2): {16-bit value, u16 staged-row byte offset}
//     entries (4 bytes) for mixed precision, {u32 offset, f32 value} (8
//     bytes) for FP32; four entries per 16-byte vector load, broadcast to the
//     lanes of a group;
//   * mixed precision (Sec. III-C): 16-bit values times 16-bit staged inputs
//     accumulate in FP32 through the mixed-precision FMA (fma.rn.f32.f16 /
//     .bf16, sm_100+); normalisation by 2^-e per slice during staging,
//     de-normalisation by 2^(e-k) in the epilogue.
#include "xct_internal.cuh"

namespace xct {
namespace {

template <class TX> struct XBytes;
template <> struct XBytes<float> { static constexpr int v = 4; };
template <> struct XBytes<__half> { static constexpr int v = 2; };
template <> struct XBytes<__nv_bfloat16> { static constexpr int v = 2; };

template <class TX, int ST>
struct Cfg {
  static constexpr int XB = XBytes<TX>::v;
  static constexpr int PIXB = ST * XB;                     // staged bytes per input row
  static constexpr int VB = PIXB >= 16 ? 16 : PIXB;        // bytes per lane load
  static constexpr int LPR = PIXB >= 128 ? 8 : PIXB / VB;  // lanes per matrix row
  static constexpr int VPL = PIXB / (VB * LPR);            // loads per lane per entry
  static constexpr int EPV = VB / XB;                      // elements per load
  static constexpr int SPL = EPV * VPL;                    // slices per lane
  static constexpr int RPW = 32 / LPR;                     // matrix rows per warp
  static constexpr int NWARPS = kRowsPerBlock / RPW;
  static constexpr int NT = NWARPS * 32;
  static constexpr bool E16 = XB == 2;
  // staging unit: 16 bytes of shared memory (or the whole row when smaller)
  static constexpr int UB = PIXB >= 16 ? 16 : PIXB;
  static constexpr int UPP = PIXB / UB;                    // units per staged row
  static constexpr int EPU = UB / XB;                      // elements per unit
  static constexpr int MIN_BLOCKS = (PIXB <= 128) ? 2 : 1;
  __host__ __device__ static size_t stage_bytes(int cap) {
    return (((size_t)cap + 1) * PIXB + 15) / 16 * 16;
  }
  static size_t smem_bytes(int cap) {
    size_t a = stage_bytes(cap) + ST * sizeof(float);
    size_t red = (size_t)NWARPS * ST * sizeof(double) + ST * sizeof(float);
    return a > red ? a : red;
  }
};

// --- shared memory vector load of VB bytes ---------------------------------
template <int VB> struct VecT;
template <> struct VecT<16> { using T = uint4; };
template <> struct VecT<8> { using T = uint2; };
template <> struct VecT<4> { using T = uint32_t; };
template <> struct VecT<2> { using T = uint16_t; };

// --- fused multiply-add of a staged vector ---------------------------------
template <class TX, int EPV> struct Fma;

template <int EPV>
struct Fma<float, EPV> {
  template <class V>
  static __device__ __forceinline__ void run(float* acc, const V& v, uint32_t wbits) {
    const float w = __uint_as_float(wbits);
    const float* x = reinterpret_cast<const float*>(&v);
#pragma unroll
    for (int e = 0; e < EPV; ++e) acc[e] = fmaf(w, x[e], acc[e]);
  }
};

template <int EPV>
struct Fma<__half, EPV> {
  template <class V>
  static __device__ __forceinline__ void run(float* acc, const V& v, uint32_t wbits) {
    const unsigned short w = (unsigned short)wbits;
    if constexpr (EPV == 1) {
      const unsigned short x = *reinterpret_cast<const unsigned short*>(&v);
      asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[0]) : "h"(x), "h"(w));
    } else {
      const uint32_t* x = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
      for (int e = 0; e < EPV / 2; ++e) {
        const unsigned short lo = (unsigned short)(x[e] & 0xffffu), hi = (unsigned short)(x[e] >> 16);
        asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e]) : "h"(lo), "h"(w));
        asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e + 1]) : "h"(hi), "h"(w));
      }
    }
  }
};

template <int EPV>
struct Fma<__nv_bfloat16, EPV> {
  template <class V>
  static __device__ __forceinline__ void run(float* acc, const V& v, uint32_t wbits) {
    const unsigned short w = (unsigned short)wbits;
    if constexpr (EPV == 1) {
      const unsigned short x = *reinterpret_cast<const unsigned short*>(&v);
      asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[0]) : "h"(x), "h"(w));
    } else {
      const uint32_t* x = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
      for (int e = 0; e < EPV / 2; ++e) {
        const unsigned short lo = (unsigned short)(x[e] & 0xffffu), hi = (unsigned short)(x[e] >> 16);
        asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * e]) : "h"(lo), "h"(w));
        asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * e + 1]) : "h"(hi), "h"(w));
      }
    }
  }
};

// --- conversion of staged inputs -------------------------------------------
template <class TX> __device__ __forceinline__ uint16_t to16(float v);
template <> __device__ __forceinline__ uint16_t to16<__half>(float v) {
  return __half_as_ushort(__float2half_rn(v));
}
template <> __device__ __forceinline__ uint16_t to16<__nv_bfloat16>(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// per-slice normalisation exponent e = ceil(log2 m) (0 for m = 0)
__device__ __forceinline__ int ceil_log2_exp(float m) {
  if (!(m > 0.0f)) return 0;
  int ex;
  float f = frexpf(m, &ex);  // m = f * 2^ex, f in [0.5, 1)
  return f == 0.5f ? ex - 1 : ex;
}

// asynchronous global -> shared copy of `bytes` (4, 8 or 16) bytes
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <class TX, int ST>
__global__ void __launch_bounds__(Cfg<TX, ST>::NT, Cfg<TX, ST>::MIN_BLOCKS)
    spmm_kernel(const int64_t* __restrict__ blk_stage, const int64_t* __restrict__ stage_pix,
                const int32_t* __restrict__ pix, const Seg* __restrict__ seg,
                const void* __restrict__ ent, int64_t nrows, int64_t ncols, int cap,
                const unsigned char* __restrict__ xs, float* __restrict__ yout,
                const uint32_t* __restrict__ in_max, int mat_scale_exp,
                double* __restrict__ dot_partial) {
  using C = Cfg<TX, ST>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const int tile = blockIdx.y;
  const int nblocks = gridDim.x;
  float* osc = reinterpret_cast<float*>(smem + C::stage_bytes(cap));  // [ST] output scales
  // staged rows of this slice tile: PIXB bytes each (16-bit normalised or FP32)
  const unsigned char* xt = xs + (size_t)tile * ncols * C::PIXB;

  for (int i = tid; i < ST; i += C::NT) {
    if (C::E16) {
      const int e = ceil_log2_exp(__uint_as_float(in_max[tile * ST + i]));
      osc[i] = ldexpf(1.0f, e - mat_scale_exp);
    } else {
      osc[i] = 1.0f;
    }
  }
  // zero slot (index cap): padding entries read it with value 0
  for (int i = tid; i < C::PIXB; i += C::NT) smem[(size_t)cap * C::PIXB + i] = 0;

  const int warp = tid >> 5, lane = tid & 31;
  const int rw = lane / C::LPR, sub = lane % C::LPR;
  const int rb = warp * C::RPW + rw;
  const int quad = rb >> 2, gq = rb & 3;

  float acc[C::SPL];
#pragma unroll
  for (int i = 0; i < C::SPL; ++i) acc[i] = 0.0f;

  const int64_t s0 = blk_stage[b], s1 = blk_stage[b + 1];
  for (int64_t s = s0; s < s1; ++s) {
    // ---- this group's segment header and first entry chunks: issued before
    // the staging copies so their latency overlaps them ----
    // Seg {int64 off; u16 cnt[4]} read as one 16-byte vector
    const uint4 sgv = __ldg(reinterpret_cast<const uint4*>(seg) + s * kQuads + quad);
    const int64_t soff = (int64_t)(((uint64_t)sgv.y << 32) | sgv.x);
    const uint32_t cw = (gq < 2) ? sgv.z : sgv.w;
    const int cnt = (int)((cw >> ((gq & 1) * 16)) & 0xffffu);
    const int nch = (cnt + 3) >> 2;   // chunks of 4 entries (padding reads slot 0.0)
    constexpr int PF = 3;             // chunks in flight
    constexpr int CW = C::E16 ? 1 : 2;        // 16-byte words per chunk of one row
    const uint4* ep = C::E16
        ? reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(ent) + soff) + gq
        : reinterpret_cast<const uint4*>(static_cast<const unsigned long long*>(ent) + soff) + gq * 2;
    uint4 pf[PF][CW];
#pragma unroll
    for (int j = 0; j < PF; ++j)
#pragma unroll
      for (int w = 0; w < CW; ++w)
        pf[j][w] = j < nch ? __ldg(ep + j * 4 * CW + w) : make_uint4(0, 0, 0, 0);

    // ---- stage the footprint rows (asynchronous byte copies) ----
    const int64_t p0 = stage_pix[s];
    const int np = (int)(stage_pix[s + 1] - p0);
    const int units = np * C::UPP;
    if constexpr (C::UB >= 4) {
      constexpr int U = 4;  // units issued per thread per round
      for (int i0 = tid; i0 < units; i0 += U * C::NT) {
        int32_t gp[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const int i = i0 + j * C::NT;
          gp[j] = i < units ? __ldg(pix + p0 + i / C::UPP) : 0;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const int i = i0 + j * C::NT;
          if (i < units) {
            const int p = i / C::UPP, u = i % C::UPP;
            cp_async<C::UB>(smem + (size_t)p * C::PIXB + u * C::UB,
                            xt + (size_t)gp[j] * C::PIXB + u * C::UB);
          }
        }
      }
      cp_async_wait_all();
    } else {
      for (int i = tid; i < units; i += C::NT)
        *reinterpret_cast<uint16_t*>(smem + (size_t)i * C::PIXB) =
            *reinterpret_cast<const uint16_t*>(xt + (size_t)__ldg(pix + p0 + i) * C::PIXB);
    }
    __syncthreads();

    // ---- multiply: this lane group's row, this stage ----
    const unsigned char* sbase = smem + sub * C::VB;
    for (int c = 0; c < nch; ++c) {
      uint4 cur[CW];
#pragma unroll
      for (int w = 0; w < CW; ++w) cur[w] = pf[0][w];
#pragma unroll
      for (int j = 0; j + 1 < PF; ++j)
#pragma unroll
        for (int w = 0; w < CW; ++w) pf[j][w] = pf[j + 1][w];
      if (c + PF < nch) {
#pragma unroll
        for (int w = 0; w < CW; ++w) pf[PF - 1][w] = __ldg(ep + (c + PF) * 4 * CW + w);
      }
      // byte offsets of the staged rows (at 128 bytes per row in the entry,
      // shifted to this tile's row size) and value bits
      constexpr int OSH = entry_shift(C::PIXB);
      uint32_t off[4], val[4];
      if constexpr (C::E16) {
        const uint32_t e4[4] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) { off[q] = e4[q] >> (16 + OSH); val[q] = e4[q] & 0xffffu; }
      } else {
        off[0] = cur[0].x >> OSH; val[0] = cur[0].y; off[1] = cur[0].z >> OSH; val[1] = cur[0].w;
        off[2] = cur[CW - 1].x >> OSH; val[2] = cur[CW - 1].y;
        off[3] = cur[CW - 1].z >> OSH; val[3] = cur[CW - 1].w;
      }
      typename VecT<C::VB>::T xv[4][C::VPL];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int v = 0; v < C::VPL; ++v)
          xv[q][v] = *reinterpret_cast<const typename VecT<C::VB>::T*>(
              sbase + off[q] + v * C::LPR * C::VB);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int v = 0; v < C::VPL; ++v)
          Fma<TX, C::EPV>::run(acc + v * C::EPV, xv[q][v], val[q]);
    }
    __syncthreads();
  }

  // ---- epilogue: de-normalise, write, per-slice squared norms ----
  const int64_t row = (int64_t)b * kRowsPerBlock + rb;
  float* yt = yout + (size_t)tile * nrows * ST;
#pragma unroll
  for (int v = 0; v < C::VPL; ++v) {
#pragma unroll
    for (int e = 0; e < C::EPV; ++e) {
      const int sl = v * C::LPR * C::EPV + sub * C::EPV + e;
      acc[v * C::EPV + e] *= osc[sl];
    }
    if (row < nrows) {
      float* dst = yt + (size_t)row * ST + v * C::LPR * C::EPV + sub * C::EPV;
      if constexpr (C::EPV % 4 == 0) {
#pragma unroll
        for (int q = 0; q < C::EPV / 4; ++q)
          reinterpret_cast<float4*>(dst)[q] =
              make_float4(acc[v * C::EPV + 4 * q], acc[v * C::EPV + 4 * q + 1],
                          acc[v * C::EPV + 4 * q + 2], acc[v * C::EPV + 4 * q + 3]);
      } else if constexpr (C::EPV == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2(acc[v * C::EPV], acc[v * C::EPV + 1]);
      } else {
        dst[0] = acc[v * C::EPV];
      }
    }
  }
  if (dot_partial != nullptr) {
    double* red = reinterpret_cast<double*>(smem);  // stage buffer is free now
    double d[C::SPL];
#pragma unroll
    for (int i = 0; i < C::SPL; ++i) d[i] = (double)acc[i] * (double)acc[i];
    // lanes with the same `sub` hold the same slices: reduce over rows
#pragma unroll
    for (int o = C::LPR; o < 32; o <<= 1) {
#pragma unroll
      for (int i = 0; i < C::SPL; ++i) d[i] += __shfl_xor_sync(0xffffffffu, d[i], o);
    }
    if (rw == 0) {
#pragma unroll
      for (int v = 0; v < C::VPL; ++v)
#pragma unroll
        for (int e = 0; e < C::EPV; ++e)
          red[warp * ST + v * C::LPR * C::EPV + sub * C::EPV + e] = d[v * C::EPV + e];
    }
    __syncthreads();
    for (int sl = tid; sl < ST; sl += C::NT) {
      double t = 0.0;
      for (int w = 0; w < C::NWARPS; ++w) t += red[w * ST + sl];
      dot_partial[(size_t)(tile * ST + sl) * nblocks + b] = t;
    }
  }
}

// FP32 [ntiles][rows][ST] -> 16-bit staging copy, slice s multiplied by
// 2^-ceil(log2 max|x_s|) before rounding to nearest even.
template <class TX, int ST>
__global__ void to_staged16_kernel(const float* __restrict__ x, uint16_t* __restrict__ out,
                                   int64_t rows, const uint32_t* __restrict__ in_max) {
  __shared__ float isc[ST];
  const int tile = blockIdx.y;
  for (int i = threadIdx.x; i < ST; i += blockDim.x)
    isc[i] = ldexpf(1.0f, -ceil_log2_exp(__uint_as_float(in_max[tile * ST + i])));
  __syncthreads();
  const int64_t n = rows * ST;
  const float* xt = x + (size_t)tile * n;
  uint16_t* ot = out + (size_t)tile * n;
  if constexpr (ST % 4 == 0) {
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i < n;
         i += (int64_t)gridDim.x * blockDim.x * 4) {
      const float4 f = *reinterpret_cast<const float4*>(xt + i);
      const int sl = (int)(i % ST);
      uint2 w;
      w.x = to16<TX>(f.x * isc[sl]) | ((uint32_t)to16<TX>(f.y * isc[sl + 1]) << 16);
      w.y = to16<TX>(f.z * isc[sl + 2]) | ((uint32_t)to16<TX>(f.w * isc[sl + 3]) << 16);
      *reinterpret_cast<uint2*>(ot + i) = w;
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      ot[i] = to16<TX>(xt[i] * isc[i % ST]);
  }
}

template <class TX, int ST>
xct_status launch(const SpmmArgs& a, cudaStream_t s) {
  using C = Cfg<TX, ST>;
  const Layout& L = *a.L;
  const size_t smem = C::smem_bytes(L.cap);
  // the opt-in shared-memory size is a per-device attribute: set it once per
  // device and size
  static std::atomic<int> configured_for[kMaxDevices];
  int cur_dev = 0;
  XCT_TRY_CUDA(cudaGetDevice(&cur_dev));
  if (cur_dev < 0 || cur_dev >= kMaxDevices || configured_for[cur_dev].load() != (int)smem + 1) {
    XCT_TRY_CUDA(cudaFuncSetAttribute(spmm_kernel<TX, ST>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (cur_dev >= 0 && cur_dev < kMaxDevices) configured_for[cur_dev].store((int)smem + 1);
  }
  if (L.nblocks == 0 || a.ntiles == 0) return XCT_OK;
  const unsigned char* src = C::E16 ? reinterpret_cast<const unsigned char*>(a.staged16)
                                    : reinterpret_cast<const unsigned char*>(a.x);
  dim3 grid((unsigned)L.nblocks, (unsigned)a.ntiles);
  spmm_kernel<TX, ST><<<grid, C::NT, smem, s>>>(L.blk_stage, L.stage_pix, L.pix, L.seg, L.ent,
                                                L.nrows, L.ncols, L.cap, src, a.y, a.in_max,
                                                a.mat_scale_exp, a.dot_partial);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

template <class TX, int ST>
xct_status launch_stage16(const SpmmArgs& a, cudaStream_t s) {
  dim3 cgrid(152 * 4, (unsigned)a.ntiles);
  to_staged16_kernel<TX, ST><<<cgrid, 256, 0, s>>>(a.x, a.staged16, a.L->ncols, a.in_max);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

template <class TX>
xct_status dispatch(const SpmmArgs& a, cudaStream_t s) {
  switch (a.st) {
    case 1: return launch<TX, 1>(a, s);
    case 2: return launch<TX, 2>(a, s);
    case 4: return launch<TX, 4>(a, s);
    case 8: return launch<TX, 8>(a, s);
    case 16: return launch<TX, 16>(a, s);
    case 32: return launch<TX, 32>(a, s);
    case 64: return launch<TX, 64>(a, s);
    default:
      set_error("slices per tile %d not supported", a.st);
      return XCT_ERR_UNSUPPORTED;
  }
}

template <class TX>
xct_status stage16(const SpmmArgs& a, cudaStream_t s) {
  switch (a.st) {
    case 1: return launch_stage16<TX, 1>(a, s);
    case 2: return launch_stage16<TX, 2>(a, s);
    case 4: return launch_stage16<TX, 4>(a, s);
    case 8: return launch_stage16<TX, 8>(a, s);
    case 16: return launch_stage16<TX, 16>(a, s);
    case 32: return launch_stage16<TX, 32>(a, s);
    case 64: return launch_stage16<TX, 64>(a, s);
    default:
      set_error("slices per tile %d not supported", a.st);
      return XCT_ERR_UNSUPPORTED;
  }
}

}  // namespace

bool spmm_supported(xct_dtype storage, int st) {
  (void)storage;
  return st == 1 || st == 2 || st == 4 || st == 8 || st == 16 || st == 32 || st == 64;
}

int pick_slices_per_tile(xct_dtype storage, int S) {
  // staged rows of 16 to 128 bytes, the widths of the persistent kernel (a
  // few slices run as 8 binary16 / 4 FP32 ones: the matrix stream, not the
  // slices, sets the time there); FP32 staged rows of 16-bit matrices at
  // least 32 bytes
  const int maxst = stages16(storage) ? 64 : 32;
  int st = stages16(storage) ? 8 : (matrix16(storage) ? 8 : 4);
  while (st < S && st < maxst) st <<= 1;
  return st;
}

xct_status spmm_stage(const SpmmArgs& a, cudaStream_t s) {
  if (!stages16(a.storage)) return XCT_OK;
  if (!a.staged16) {
    set_error("16-bit storage needs a staging buffer");
    return XCT_ERR_INVALID;
  }
  if (a.L->ncols == 0 || a.ntiles == 0) return XCT_OK;
  return a.storage == XCT_F16 ? stage16<__half>(a, s) : stage16<__nv_bfloat16>(a, s);
}

xct_status spmm_run(const SpmmArgs& a0, cudaStream_t s) {
  const SpmmArgs a = on_product_layout(a0);
  const int max_cap = 65535 / a.L->unit - 1;   // the zero slot's offset fits 16 bits
  if (a.L->cap > max_cap) {
    set_error("stage capacity %d exceeds the 16-bit staged-row offset (at most %d)", a.L->cap,
              max_cap);
    return XCT_ERR_UNSUPPORTED;
  }
  if (!valid_storage(a.storage)) {
    set_error("unknown storage type");
    return XCT_ERR_INVALID;
  }
  if (spmm_pipe_applies(a)) return spmm_pipe(a, s);
  if (a.L->unit != kEntryRowBytes || a.L->pair) {
    set_error("wide-stage or paired layout without a fitting persistent product");
    return XCT_ERR_UNSUPPORTED;
  }
  if (matrix16(a.storage) && !stages16(a.storage)) {
    set_error("16-bit matrix with FP32 vectors needs the persistent product (tile width %d, "
              "stage capacity %d)", a.st, a.L->cap);
    return XCT_ERR_UNSUPPORTED;
  }
  switch (a.storage) {
    case XCT_F32: return dispatch<float>(a, s);
    case XCT_F16: return dispatch<__half>(a, s);
    default: return dispatch<__nv_bfloat16>(a, s);
  }
}

xct_status spmm(const SpmmArgs& a, cudaStream_t s) {
  XCT_TRY(spmm_stage(a, s));
  return spmm_run(a, s);
}

int spmm_dot_count(const SpmmArgs& a) { return a.L->nblocks; }

}  // namespace xct

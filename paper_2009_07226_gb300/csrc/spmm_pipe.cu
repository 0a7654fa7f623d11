// Persistent, warp-specialised form of the fused product Y = M X (paper
// Sec. III-B: input buffering, register reuse, output buffering, multi-stage
// buffering; Sec. III-C: mixed precision).
//
// A producer warp takes blocks of 64 rows from a work counter and streams
// each stage of each block into one of two shared-memory buffers with bulk
// asynchronous copies (cp.async.bulk) counted in bytes on the buffer's
// mbarrier: one copy per contiguous run of the stage's staged input rows
// (runs of consecutive Hilbert ids, with gaps of a few unreferenced rows
// filled in by the plan so that runs are longer; the run list itself
// arrives one stage ahead by another bulk copy) and one for the stage's
// packed entries.  Each copy costs the TMA unit a fixed time whatever its
// size, so the segment headers (256 B) go through the producer's registers
// instead.  The consumer warps (16
// for 128-byte staged rows, 8 for 64-byte, 4 for 32-byte; 2, 3 or 4 CTAs per
// SM) compute from shared memory only and release the buffer through a
// second mbarrier; while they work on one stage the next one (possibly of the
// next block) is already in flight.  The lane layout of the consumers is the
// one of spmm.cu: a group of lanes holds different slices of one row, so every
// shared-memory wavefront reads one contiguous staged row.
//
// Staged rows are 16-bit (normalised per slice) or FP32; matrix values are
// FP32 or 16-bit (see PCfg and PFma).
//
// Every wait is bounded (xct_set_wait_limit, 2 s by default); a wait that
// runs out sets the caller's error flag, waits (bounded) for the copies this
// CTA has in flight and returns.  The consumers' block-end rendezvous is an
// mbarrier too, so no warp can be left at an unbounded barrier.
#include <type_traits>

#include "xct_internal.cuh"

namespace xct {
namespace {

template <class TX> struct PBytes;
template <> struct PBytes<float> { static constexpr int v = 4; };
template <> struct PBytes<__half> { static constexpr int v = 2; };
template <> struct PBytes<__nv_bfloat16> { static constexpr int v = 2; };

// TX: type of the staged input rows; TW: type of the stored matrix values
template <class TX, class TW, int ST>
struct PCfg {
  static constexpr int XB = PBytes<TX>::v;
  static constexpr int PIXB = ST * XB;
  static constexpr int VB = 16;
  static constexpr bool X16 = XB == 2;             // normalised 16-bit staged rows
  static constexpr int LPR = PIXB >= 128 ? (X16 ? 4 : 8) : PIXB / 16;   // lanes holding slices of a row
  // lanes splitting a row's chunks of 4 entries (lane e takes 4 / ES
  // consecutive entries of every chunk; their partial sums are added at the
  // block end): 16-byte staged rows keep 8 consumer warps per block this way
  // instead of 2; 128-byte rows of 16-bit slices give each lane 16 slices
  // of a row (two 16-byte vectors per entry), so the per-entry work
  // (offset, address, entry load) is shared by twice the FMAs (1.4% faster
  // binary16 products; FP32 rows measured slower this way and keep 8 lanes
  // of 4 slices)
  static constexpr int ES = PIXB == 16 ? 4 : (PIXB >= 128 && X16 ? 2 : 1);
  static constexpr int VPL = PIXB / (VB * LPR);
  // with two lanes per row and two vectors per lane, lane e reads half e of
  // the staged row first, so the two rows a quarter warp reads at once fall
  // in different banks; its accumulators acc[0 .. EPV) hold half e
  static constexpr bool SWZ = ES == 2 && VPL == 2;
  static constexpr int EPV = VB / XB;
  static constexpr int SPL = EPV * VPL;
  static constexpr int RPW = 32 / (LPR * ES);
  static constexpr int NC = kRowsPerBlock / RPW;   // consumer warps
  static constexpr int NT = (NC + 1) * 32;         // + one producer warp
  static constexpr bool W16 = PBytes<TW>::v == 2;  // {u16 index, 16-bit value} entries
  static constexpr int EB = W16 ? 4 : 8;           // bytes per packed entry
  static constexpr int OSH = entry_shift(PIXB);    // entry offset -> this row size
  static constexpr int NB = PIXB == 16 ? kPipeBufs16 : kPipeBufs;   // stage buffers
  // CTAs per SM: narrower staged rows mean fewer consumer warps per CTA
  // and smaller stage buffers, so more CTAs share an SM
  static constexpr int MINB = PIXB >= 128 ? 2 : (PIXB == 64 ? 3 : (PIXB == 16 ? kPipeMinb16 : 4));
};

// stage descriptors are requested this many stages before the stage's
// copies, into kDescSlots = kDescAhead + 1 slots
constexpr int kDescAhead = 3;
constexpr int kDescSlots = kDescAhead + 1;

struct __align__(16) Hdr {
  int32_t work;    // work item inside its product (tile * nblocks + block), -1 = no more work
  int32_t kstage;  // stage index inside the block
  int32_t last;    // last stage of the block
  int32_t np;      // staged rows (0: a block without entries)
  int32_t prod;    // product index in the launch
  int32_t pad[3];
};

// One product of a launch: a layout with its input / output vectors.
struct PipeLayout {
  const int64_t* blk_stage;
  const unsigned char* desc;  // [nstages] stage descriptors (StageDescHead ...)
  int64_t desc_bytes;
  const unsigned char* ent;
  int64_t nrows, ncols;
  int cap, nblocks, ntiles;
  int work_begin;            // first work item of this product in the launch
  const unsigned char* xs;   // staged rows [tile][ncols][PIXB bytes]
  float* y;                  // [tile][nrows][ST]
  const uint32_t* in_max;
  int mat_scale_exp;
  double* dot;               // [ntiles*ST][nblocks] or null
};

struct PipeArgs {
  PipeLayout L[kMaxPipeProducts];
  int nl;                    // products in this launch
  int nwork;                 // work items over all products
  int cap;                   // largest stage capacity (buffer rows)
  uint32_t dbytes;           // per-slot descriptor region (128-byte multiple)
  int* work;
  int* err;
  uint32_t xbytes, ebytes;   // per-buffer region sizes (128-byte multiples)
  uint64_t wait_ns;          // limit of every pipeline wait
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(tx)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(tx)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking test of the phase of `parity`
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of `parity` to complete; false once `limit_ns` of wall
// time has passed without it (checked every 256 tries; a limit of 0 only
// tests the phase once, without suspending).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return mbar_test(bar, parity);   // no waiting at all
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255u) == 0 && now_ns() - t0 > limit_ns) return false;
  }
}
// the limit of the waits that let copies already issued land before a CTA
// that gave up exits (independent of the configurable limit)
constexpr uint64_t kDrainNs = 2000000000ull;
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

// a hint to bring `bytes` (a multiple of 16) at `src` (16-byte aligned) into
// L2; nothing waits for it
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// FMA of one staged 16-byte vector by one matrix value.  FP32 staged rows:
// the value converted once (exactly), then pairs of slices through the
// packed FP32 FMA (each half rounds like fmaf; measured 5% faster than
// scalar FMAs).  16-bit staged rows: the mixed-precision FMA (16-bit
// operands, FP32 accumulator), which measured faster than converting the
// operands and using packed FMAs (1.66 vs 2.31 ms for the binary16
// projection of 512^2 x 768 angles x 512 bins x 64 slices).
__device__ __forceinline__ void ffma2(float* acc, float2 w, float2 x) {
  float2 c = make_float2(acc[0], acc[1]);
  c = __ffma2_rn(w, x, c);
  acc[0] = c.x;
  acc[1] = c.y;
}
template <int EPV>
__device__ __forceinline__ void ffma2_row(float* acc, float w, const uint4& v) {
  const float* x = reinterpret_cast<const float*>(&v);
#pragma unroll
  for (int e = 0; e < EPV / 2; ++e)
    ffma2(acc + 2 * e, make_float2(w, w), make_float2(x[2 * e], x[2 * e + 1]));
}
template <class TX, class TW, int EPV> struct PFma;
template <int EPV> struct PFma<float, float, EPV> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t wbits) {
    ffma2_row<EPV>(acc, __uint_as_float(wbits), v);
  }
};
template <int EPV> struct PFma<float, __half, EPV> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t wbits) {
    ffma2_row<EPV>(acc, __half2float(__ushort_as_half((unsigned short)wbits)), v);
  }
};
template <int EPV> struct PFma<float, __nv_bfloat16, EPV> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t wbits) {
    ffma2_row<EPV>(acc, __uint_as_float((wbits & 0xffffu) << 16), v);
  }
};
// 16-bit staged rows: one mixed-precision FMA per slice, each its own
// instruction with 16-bit operands split from the 32-bit words in C (ptxas
// then takes the halves in place: 5% fewer instructions and 2.5% faster
// products than splitting both halves inside one asm block)
template <int EPV> struct PFma<__half, __half, EPV> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t wbits) {
    const unsigned short w = (unsigned short)wbits;
    const uint32_t* x = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
    for (int e = 0; e < EPV / 2; ++e) {
      const unsigned short lo = (unsigned short)(x[e] & 0xffffu), hi = (unsigned short)(x[e] >> 16);
      asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e]) : "h"(lo), "h"(w));
      asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc[2 * e + 1]) : "h"(hi), "h"(w));
    }
  }
};
template <int EPV> struct PFma<__nv_bfloat16, __nv_bfloat16, EPV> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t wbits) {
    const unsigned short w = (unsigned short)wbits;
    const uint32_t* x = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
    for (int e = 0; e < EPV / 2; ++e) {
      const unsigned short lo = (unsigned short)(x[e] & 0xffffu), hi = (unsigned short)(x[e] >> 16);
      asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * e]) : "h"(lo), "h"(w));
      asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc[2 * e + 1]) : "h"(hi), "h"(w));
    }
  }
};

// A shared slot of a paired layout: one 16-byte vector of a staged row (8
// slices) times the values of both rows of a pair; acc[0 .. 8) and
// acc[8 .. 16) are the two rows' sums of the same 8 slices (two plain
// vector FMAs: measured faster than one asm block feeding both rows).
template <class TX> struct PFma2;
template <> struct PFma2<__half> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t w0bits, uint32_t w1bits) {
    PFma<__half, __half, 8>::run(acc, v, w0bits);
    PFma<__half, __half, 8>::run(acc + 8, v, w1bits);
  }
};
template <> struct PFma2<__nv_bfloat16> {
  static __device__ __forceinline__ void run(float* acc, const uint4& v, uint32_t w0bits, uint32_t w1bits) {
    PFma<__nv_bfloat16, __nv_bfloat16, 8>::run(acc, v, w0bits);
    PFma<__nv_bfloat16, __nv_bfloat16, 8>::run(acc + 8, v, w1bits);
  }
};

// staged-row byte offset (at 128 bytes per row) and value bits of one packed
// entry: {16-bit value, u16 offset} or {u32 offset, f32 value}
__device__ __forceinline__ uint32_t eoff(uint32_t e) { return e >> 16; }
__device__ __forceinline__ uint32_t eval(uint32_t e) { return e & 0xffffu; }
__device__ __forceinline__ uint32_t eoff(uint2 e) { return e.x; }
__device__ __forceinline__ uint32_t eval(uint2 e) { return e.y; }

__device__ __forceinline__ int ceil_log2_exp_p(float m) {
  if (!(m > 0.0f)) return 0;
  int ex;
  const float f = frexpf(m, &ex);
  return f == 0.5f ? ex - 1 : ex;
}

// An unevaluated sum h + l of two FP32 values: squares of FP32 values are
// exact in it (l from an FMA), and sums of such non-negative terms keep
// about 47 bits (two-sum of the high parts, then renormalisation), on the
// FP32 pipes.
struct Ff {
  float h, l;
};
__device__ __forceinline__ Ff ff_square(float r) {
  const float h = __fmul_rn(r, r);
  return {h, __fmaf_rn(r, r, -h)};
}
__device__ __forceinline__ Ff sum2(Ff a, Ff b) {
  const float s = __fadd_rn(a.h, b.h);
  const float v = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));   // s's error, exact
  const float t = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ double sum2(double a, double b) { return a + b; }
__device__ __forceinline__ Ff shfl_xor(Ff v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

// Sum over the rows of a warp of N values per lane (FP64 or Ff), lanes
// paired over lane bits O, 2 O, .. 16: while a lane holds more than one
// value, the pair splits them (the lane with bit O clear keeps the first
// half, its partner the second; each adds the partner's value of the same
// slice), so every addition is done once; a single value goes through the
// plain butterfly.  Each slice's sum is the same tree of additions as the
// plain butterfly (both additions are commutative bit for bit).
// `base` returns the index (among the lane's N) of its first kept value.
template <int N, int O, class T>
__device__ __forceinline__ void halve_rows(T* d, int lane, int& base) {
  if constexpr (O < 32) {
    if constexpr (N > 1) {
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const T send = up ? d[i] : d[N / 2 + i];
        const T keep = up ? d[N / 2 + i] : d[i];
        d[i] = sum2(keep, shfl_xor(send, O));
      }
      if (up) base += N / 2;
      halve_rows<N / 2, 2 * O>(d, lane, base);
    } else {
      d[0] = sum2(d[0], shfl_xor(d[0], O));
      halve_rows<1, 2 * O>(d, lane, base);
    }
  }
}
// values a lane holds after halve_rows<N, O>, and the lane bits over which
// lanes then hold duplicates (the plain butterfly's levels)
__host__ __device__ constexpr int halved_count(int n, int o) { return o >= 32 ? n : halved_count(n > 1 ? n / 2 : 1, 2 * o); }
__host__ __device__ constexpr int halved_dup_mask(int n, int o) {
  return o >= 32 ? 0 : (n > 1 ? halved_dup_mask(n / 2, 2 * o) : (o | halved_dup_mask(1, 2 * o)));
}

template <class TX, class TW, int ST, bool WIDE, bool PAIR>
__global__ void __launch_bounds__(PCfg<TX, TW, ST>::NT, PCfg<TX, TW, ST>::MINB)
    spmm_pipe_kernel(PipeArgs a) {
  using C = PCfg<TX, TW, ST>;
  // paired layouts: 128-byte rows of 16-bit slices, 8-byte slots
  static_assert(!PAIR || (C::X16 && C::W16 && C::PIXB == 128 && C::SWZ && !WIDE), "paired layout");
  constexpr int EB = PAIR ? 8 : C::EB;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bufbytes = a.xbytes + a.ebytes + 256 + 128;
  constexpr int NB = C::NB;
  constexpr int DS = kDescSlots;
  // [NB stage buffers][DS descriptor slots][barriers][DS stage identities]
  unsigned char* dslots = smem + NB * bufbytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(dslots + DS * a.dbytes);
  uint64_t* empty = full + NB;
  uint64_t* dbar = full + 2 * NB;        // descriptor of a stage landed
  uint64_t* redbar = full + 2 * NB + DS;  // consumers' rendezvous at a block end (2)
  int4* ident = reinterpret_cast<int4*>(redbar + 2);
  // 16-byte rows of 16-bit slices: [NB][NC][ST] block-end partials (FP32
  // pairs) and [NB] counters of the warps past a block end
  float2* dpair = reinterpret_cast<float2*>(ident + DS);
  int* dcnt = reinterpret_cast<int*>(dpair + (C::PIXB == 16 && C::X16 ? NB * C::NC * ST : 0));
  auto dslot = [&](int k) { return dslots + (size_t)k * a.dbytes; };
  auto xbuf = [&](int b) { return smem + b * bufbytes; };
  auto ebuf = [&](int b) { return smem + b * bufbytes + a.xbytes; };
  auto sbuf = [&](int b) { return smem + b * bufbytes + a.xbytes + a.ebytes; };
  auto hbuf = [&](int b) { return reinterpret_cast<Hdr*>(smem + b * bufbytes + a.xbytes + a.ebytes + 256); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < NB; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], C::NC);
    }
    for (int k = 0; k < kDescSlots; ++k) mbar_init(&dbar[k], 1);
    mbar_init(&redbar[0], C::NC);
    mbar_init(&redbar[1], C::NC);
    if constexpr (C::PIXB == 16 && C::X16)
      for (int b = 0; b < NB; ++b) dcnt[b] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero slot of each product (row `cap` of its layout) in every buffer:
  // padding entries read it with value 0
  for (int l = 0; l < a.nl; ++l)
    for (int i = tid; i < C::PIXB; i += C::NT)
      for (int b = 0; b < NB; ++b) xbuf(b)[(size_t)a.L[l].cap * C::PIXB + i] = 0;
  __syncthreads();

  const int nwork = a.nwork;

  if (warp == C::NC) {
    // ----------------------------- producer -----------------------------
    // A cursor walks the stages of the CTA's blocks: work item of the launch
    // (-1: no more), its product and work item inside the product, stage
    // index in its block, stages in the block, layout stage (-1 for a block
    // without entries).  Each stage's descriptor (one bulk copy from an
    // array of fixed stride, so its address needs only the stage index) is
    // requested kDescAhead stages before the stage's copies are issued, and
    // the next block is claimed from the work counter one block ahead (lane
    // 0 holds the counter's answer until it is needed): no metadata load is
    // on the path of a stage.
    struct Cursor {
      int w, l, wl, k, nst, s;
    };
    struct Claim {
      int raw;      // lane 0: the work counter's answer
      int age;      // stages since the claim
      bool resolved;
      int w, l, wl;
      int64_t s0, s1;
    };
    auto claim = [&]() -> Claim {
      Claim c{0, 0, false, -1, 0, 0, 0, 0};
      if (lane == 0) c.raw = atomicAdd(a.work, 1);
      return c;
    };
    auto resolve = [&](Claim& c) {
      if (c.resolved) return;
      c.resolved = true;
      c.w = __shfl_sync(0xffffffffu, c.raw, 0);
      if (c.w >= nwork) {
        c.w = -1;
        return;
      }
      int l = a.nl - 1;
      while (l > 0 && c.w < a.L[l].work_begin) --l;
      const PipeLayout& P = a.L[l];
      c.l = l;
      c.wl = c.w - P.work_begin;
      const int b = c.wl % P.nblocks;
      c.s0 = P.blk_stage[b];
      c.s1 = P.blk_stage[b + 1];
    };
    auto start_of = [&](const Claim& c) -> Cursor {
      if (c.w < 0) return Cursor{-1, 0, 0, 0, 1, -1};
      return Cursor{c.w, c.l, c.wl, 0, c.s1 > c.s0 ? (int)(c.s1 - c.s0) : 1,
                    c.s1 > c.s0 ? (int)c.s0 : -1};
    };
    Claim pend = claim();
    resolve(pend);
    Cursor cur = start_of(pend);
    if (pend.w >= 0) pend = claim();
    auto advance = [&](Cursor& c) {
      if (c.w < 0) return;
      if (c.k + 1 < c.nst) {
        ++c.k;
        if (c.s >= 0) ++c.s;
        return;
      }
      resolve(pend);
      c = start_of(pend);
      if (pend.w >= 0) pend = claim();
    };
    // the descriptor of the cursor's stage into slot k, with the stage's
    // identity (work item in its product or -1, product, stage in block,
    // flags: 1 = last stage of its block, 2 = has entries)
    auto request = [&](const Cursor& c, int k) {
      if (lane != 0) return;
      const bool real = c.w >= 0 && c.s >= 0;
      ident[k] = make_int4(c.w >= 0 ? c.wl : -1, c.l, c.k,
                           (c.k == c.nst - 1 ? 1 : 0) | (real ? 2 : 0));
      if (real) {
        const PipeLayout& P = a.L[c.l];
        mbar_arrive_tx(&dbar[k], (uint32_t)P.desc_bytes);
        bulk_g2s(dslot(k), P.desc + (size_t)c.s * P.desc_bytes, (uint32_t)P.desc_bytes, &dbar[k]);
      } else {
        mbar_arrive(&dbar[k]);
      }
    };
    bool ok = true;
    uint32_t fail_it = 0, req_hi = 0;   // req_hi: last stage whose descriptor was requested
    for (int j = 0; j < kDescAhead; ++j) {
      request(cur, j);
      advance(cur);
    }
    req_hi = kDescAhead - 1;
    for (uint32_t it = 0;; ++it) {
      const int buf = (int)(it % NB);
      const uint32_t use = it / NB;
      const int ds = (int)(it % DS);
      // the claim made at the last block crossing: its answer has had two
      // stages to arrive
      if (!pend.resolved && ++pend.age >= 2) resolve(pend);
      // slot (it + kDescAhead) % DS last held stage it - 1, read by now;
      // this warp's reads of it precede the copy into it
      __syncwarp();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      request(cur, (int)((it + kDescAhead) % DS));
      req_hi = it + kDescAhead;
      advance(cur);
      if (!mbar_wait(&dbar[ds], (it / DS) & 1, a.wait_ns)) { ok = false; fail_it = it; break; }
      __syncwarp();
      const int4 id = ident[ds];
      const bool real = (id.w & 2) != 0;
      const PipeLayout& P = a.L[id.y];
      const unsigned char* dd = dslot(ds);
      const StageDescHead dh = *reinterpret_cast<const StageDescHead*>(dd);
      const int np = real ? (int)dh.np : 0;
      const uint32_t eb = real ? dh.slots * (uint32_t)EB : 0u;
      // a wide stage's entries, read by the consumers from global memory
      // about two stages from now, are brought into L2 before this warp
      // waits for the buffer (measured 3.5% faster than no prefetch)
      if (WIDE && lane == 0 && eb) bulk_prefetch_l2(P.ent + (size_t)dh.e0 * EB, eb);
      if (!mbar_wait(&empty[buf], (use & 1) ^ 1, a.wait_ns)) { ok = false; fail_it = it; break; }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) {
        Hdr h;
        h.work = id.x;
        h.prod = id.y;
        h.kstage = id.z;
        h.last = id.w & 1;
        h.np = np;
        *hbuf(buf) = h;
      }
      if (real) {
        const int tile = id.x / P.nblocks;
        const unsigned char* xt = P.xs + (size_t)tile * P.ncols * C::PIXB;
        // one bulk copy per contiguous run of staged rows, plus the stage's
        // packed entries, all counted in bytes on the full barrier (the
        // expected count is set before any copy starts)
        // (a wide-stage layout's entries stay in global memory)
        if (lane == 0) mbar_expect_tx(&full[buf], (uint32_t)np * C::PIXB + (WIDE ? 0u : eb));
        // the segment headers, from the descriptor, by plain stores (the
        // full barrier's arrival below publishes them with the header)
        reinterpret_cast<uint2*>(sbuf(buf))[lane] =
            reinterpret_cast<const uint2*>(dd + sizeof(StageDescHead))[lane];
        __syncwarp();
        const int2* rl = reinterpret_cast<const int2*>(dd + sizeof(StageDescHead) + kQuads * 16);
        unsigned char* xd = xbuf(buf);
        for (int k = lane; k < (int)dh.nr; k += 32) {
          const int2 run = rl[k];
          if (run.x >= 0) {
            const uint32_t len = (uint32_t)(rl[k + 1].y - run.y);
            bulk_g2s(xd + (size_t)run.y * C::PIXB, xt + (size_t)run.x * C::PIXB, len * C::PIXB,
                     &full[buf]);
          }
        }
        if (!WIDE && lane == 0 && eb) bulk_g2s(ebuf(buf), P.ent + (size_t)dh.e0 * EB, eb, &full[buf]);
      }
      // the single arrival of this phase; it also publishes the header
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[buf]);
      if (id.x < 0) break;
    }
    if (!ok) {
      if (lane == 0) atomicExch(a.err, 1);
      // let copies already issued land before the CTA's shared memory goes
      // away: the stage copies of the last NB iterations before the failing
      // one (every iteration arrives on its full barrier, with copies or
      // without), and the descriptors requested for stages fail_it to req_hi
      // (every request completes a phase of its slot's barrier)
      for (uint32_t j = fail_it > (uint32_t)NB ? fail_it - NB : 0; j < fail_it; ++j)
        mbar_wait(&full[j % NB], (j / NB) & 1, kDrainNs);
      for (uint32_t j = fail_it; j <= req_hi; ++j) mbar_wait(&dbar[j % DS], (j / DS) & 1, kDrainNs);
    }
    return;
  }

  // ------------------------------ consumers ------------------------------
  const int rw = lane / (C::LPR * C::ES), el = (lane / C::LPR) % C::ES, sub = lane % C::LPR;
  const int rb = warp * C::RPW + rw;
  const int quad = rb >> 2, gq = rb & 3;
  float acc[C::SPL];
#pragma unroll
  for (int i = 0; i < C::SPL; ++i) acc[i] = 0.0f;
  uint32_t rphase = 0;   // phase of the block-end rendezvous barriers
  int live = 8;   // wide stages: live slices of the block's tile (2, 4 or 8)
  for (uint32_t it = 0;; ++it) {
    const int buf = (int)(it % NB);
    if (!mbar_wait(&full[buf], (it / NB) & 1, a.wait_ns)) {
      if (lane == 0) atomicExch(a.err, 1);
      return;
    }
    const Hdr h = *hbuf(buf);
    if (h.work < 0) break;
    if (h.kstage == 0) {
#pragma unroll
      for (int i = 0; i < C::SPL; ++i) acc[i] = 0.0f;
      if constexpr (WIDE) {
        // live slices of the block's tile: 2 when slices 2 .. 7 are all
        // zero (one or two slices, the rest padding), 4 when slices 4 .. 7
        // are, else 8; only their bytes of each staged row are read
        const uint32_t* im = a.L[h.prod].in_max + (h.work / a.L[h.prod].nblocks) * ST;
        const uint32_t hi4 = __ldg(im + 4) | __ldg(im + 5) | __ldg(im + 6) | __ldg(im + 7);
        live = hi4 != 0u ? 8 : ((__ldg(im + 2) | __ldg(im + 3)) != 0u ? 4 : 2);
      }
    }
    if (h.np > 0) {
      const uint4 sgv = *reinterpret_cast<const uint4*>(sbuf(buf) + quad * 16);
      const uint4 sg0 = *reinterpret_cast<const uint4*>(sbuf(buf));
      const int64_t off = (int64_t)(((uint64_t)sgv.y << 32) | sgv.x);
      const int64_t base = (int64_t)(((uint64_t)sg0.y << 32) | sg0.x);
      const uint32_t cw = (gq < 2) ? sgv.z : sgv.w;
      const int cnt = (int)((cw >> ((gq & 1) * 16)) & 0xffffu);
      const int nch = (cnt + 3) >> 2;
      const unsigned char* xs = xbuf(buf) + sub * C::VB;
      if constexpr (PAIR) {
        // paired layout (placement described with kPairUA): lane 16 p + 8 e
        // + j holds slices 8 j .. 8 j + 7 of both rows of pair p and takes
        // the pair's slots of lane index e; the 8 lanes of a quarter warp
        // read one whole 128-byte staged row per slot
        static_assert(kPairUA == 4 && kPairUB == 2, "slot loads below");
        const int pp = lane >> 4, pe = (lane >> 3) & 1;
        const uint32_t cwp = pp ? sgv.w : sgv.z;
        const int nsc = (int)(cwp & 0xffffu), nxc = (int)(cwp >> 16);
        const int s0c = (int)(sgv.z & 0xffffu), s1c = (int)(sgv.w & 0xffffu);
        const int ga = ((s0c > s1c ? s0c : s1c) + kPairUA - 1) / kPairUA;
        const uint2* eq = reinterpret_cast<const uint2*>(ebuf(buf) + (off - base) * EB);
        const unsigned char* xp = xbuf(buf) + (lane & 7) * C::VB;
        // shared slots: one staged-row vector for both rows
        const uint2* ea = eq + (2 * pp + pe) * kPairUA;
        int c = 0;
        for (; c + kPairUA <= nsc; c += kPairUA) {
          const uint4* e4 = reinterpret_cast<const uint4*>(ea + c * 4);
          const uint4 u0 = e4[0], u1 = e4[1];
          const uint32_t ex[4] = {u0.x, u0.z, u1.x, u1.z};
          const uint32_t ey[4] = {u0.y, u0.w, u1.y, u1.w};
          uint4 xv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = *reinterpret_cast<const uint4*>(xp + (ex[q] >> 16));
#pragma unroll
          for (int q = 0; q < 4; ++q) PFma2<TX>::run(acc, xv[q], ex[q], ey[q]);
        }
        for (; c < nsc; ++c) {
          const uint2 ev = ea[(c / kPairUA) * 4 * kPairUA + c % kPairUA];
          PFma2<TX>::run(acc, *reinterpret_cast<const uint4*>(xp + (ev.x >> 16)), ev.x, ev.y);
        }
        // split slots: one column of each row
        const uint2* ebp = eq + ga * 4 * kPairUA + (2 * pp + pe) * kPairUB;
        for (c = 0; c + kPairUB <= nxc; c += kPairUB) {
          const uint4 u = *reinterpret_cast<const uint4*>(ebp + c * 4);
          const uint32_t ex[2] = {u.x, u.z}, ey[2] = {u.y, u.w};
          uint4 x0[2], x1[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            x0[q] = *reinterpret_cast<const uint4*>(xp + (ex[q] >> 16));
            x1[q] = *reinterpret_cast<const uint4*>(xp + (ey[q] >> 16));
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            PFma<TX, TW, C::EPV>::run(acc, x0[q], ex[q] & 0xffffu);
            PFma<TX, TW, C::EPV>::run(acc + C::EPV, x1[q], ey[q] & 0xffffu);
          }
        }
        for (; c < nxc; ++c) {
          const uint2 ev = ebp[(c / kPairUB) * 4 * kPairUB + c % kPairUB];
          PFma<TX, TW, C::EPV>::run(acc, *reinterpret_cast<const uint4*>(xp + (ev.x >> 16)), ev.x & 0xffffu);
          PFma<TX, TW, C::EPV>::run(acc + C::EPV, *reinterpret_cast<const uint4*>(xp + (ev.y >> 16)),
                                    ev.y & 0xffffu);
        }
      } else if constexpr (WIDE) {
        // wide stages: the row's chunks of 4 entries are read straight from
        // global memory (16 bytes per lane, two chunks in flight ahead of
        // the one in use); lane e of the row takes chunks e, e + 4, ...;
        // the quad's chunks lie in groups of 4 per row, all 4 rows' groups
        // together, so the 8 lanes of two rows read 128 contiguous bytes
        // (group i of row gq at 16 i + 4 gq); offsets address 16-byte staged
        // rows directly
        const uint4* gp =
            reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(a.L[h.prod].ent) + off) +
            gq * 4 + el;
        const uint4 z = make_uint4(0, 0, 0, 0);
        // (with 2 or 4 live slices, 4 or 8 bytes of the row and 2 or 4 FMAs
        // per entry: the other slices' accumulators stay zero)
        auto rows = [&](auto live) {
          constexpr int LV = decltype(live)::value;
          int k = el;
          uint4 n0 = k < nch ? __ldg(gp) : z;
          uint4 n1 = k + 4 < nch ? __ldg(gp + 16) : z;
          const uint4* pn = gp + 32;
          for (; k < nch; k += 4) {
            const uint4 cur = n0;
            n0 = n1;
            n1 = k + 8 < nch ? __ldg(pn) : z;
            pn += 16;
            const uint32_t e4[4] = {cur.x, cur.y, cur.z, cur.w};
            uint4 xv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if constexpr (LV == 2) {
                xv[q] = make_uint4(*reinterpret_cast<const uint32_t*>(xs + (e4[q] >> 16)), 0u, 0u, 0u);
              } else if constexpr (LV == 4) {
                const uint2 v = *reinterpret_cast<const uint2*>(xs + (e4[q] >> 16));
                xv[q] = make_uint4(v.x, v.y, 0u, 0u);
              } else
                xv[q] = *reinterpret_cast<const uint4*>(xs + (e4[q] >> 16));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) PFma<TX, TW, LV>::run(acc, xv[q], e4[q] & 0xffffu);
          }
        };
        if (live == 2)
          rows(std::integral_constant<int, 2>{});
        else if (live == 4)
          rows(std::integral_constant<int, 4>{});
        else
          rows(std::integral_constant<int, C::EPV>{});
      } else if constexpr (C::ES > 1) {
        // EPL entries of each chunk per lane; four entries in flight per step
        constexpr int EPL = 4 / C::ES;
        constexpr int U = 4 / EPL;   // chunks per step
        using E = typename std::conditional<C::W16, uint32_t, uint2>::type;
        const E* ep = reinterpret_cast<const E*>(ebuf(buf) + (off - base) * C::EB) + gq * 4 + el * EPL;
        const unsigned char* x0 = xs + (C::SWZ ? el : 0) * C::LPR * C::VB;
        const unsigned char* x1 = xs + (C::SWZ ? 1 - el : 1) * C::LPR * C::VB;
        int c = 0;
        for (; c + U <= nch; c += U) {
          E ev[4];
          uint4 xa[4], xb[4];
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < EPL; ++j) ev[u * EPL + j] = ep[(c + u) * 16 + j];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t o = eoff(ev[q]) >> C::OSH;
            xa[q] = *reinterpret_cast<const uint4*>(x0 + o);
            if constexpr (C::VPL == 2) xb[q] = *reinterpret_cast<const uint4*>(x1 + o);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            PFma<TX, TW, C::EPV>::run(acc, xa[q], eval(ev[q]));
            if constexpr (C::VPL == 2) PFma<TX, TW, C::EPV>::run(acc + C::EPV, xb[q], eval(ev[q]));
          }
        }
        for (; c < nch; ++c) {
#pragma unroll
          for (int j = 0; j < EPL; ++j) {
            const E ev = ep[c * 16 + j];
            const uint32_t o = eoff(ev) >> C::OSH;
            PFma<TX, TW, C::EPV>::run(acc, *reinterpret_cast<const uint4*>(x0 + o), eval(ev));
            if constexpr (C::VPL == 2)
              PFma<TX, TW, C::EPV>::run(acc + C::EPV, *reinterpret_cast<const uint4*>(x1 + o), eval(ev));
          }
        }
      } else if constexpr (C::W16) {
        const uint4* ep = reinterpret_cast<const uint4*>(ebuf(buf) + (off - base) * 4) + gq;
        uint4 nx = nch > 0 ? ep[0] : make_uint4(0, 0, 0, 0);
        for (int c = 0; c < nch; ++c) {
          const uint4 cur = nx;
          if (c + 1 < nch) nx = ep[(c + 1) * 4];
          const uint32_t e4[4] = {cur.x, cur.y, cur.z, cur.w};
          uint4 xv[4][C::VPL];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < C::VPL; ++v)
              xv[q][v] = *reinterpret_cast<const uint4*>(xs + (e4[q] >> (16 + C::OSH)) +
                                                         v * C::LPR * C::VB);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < C::VPL; ++v)
              PFma<TX, TW, C::EPV>::run(acc + v * C::EPV, xv[q][v], e4[q] & 0xffffu);
        }
      } else {
        const uint4* ep = reinterpret_cast<const uint4*>(ebuf(buf) + (off - base) * 8) + gq * 2;
        uint4 na = make_uint4(0, 0, 0, 0), nb = na;
        if (nch > 0) { na = ep[0]; nb = ep[1]; }
        for (int c = 0; c < nch; ++c) {
          const uint4 ca = na, cb = nb;
          if (c + 1 < nch) { na = ep[(c + 1) * 8]; nb = ep[(c + 1) * 8 + 1]; }
          const uint32_t idx[4] = {ca.x, ca.z, cb.x, cb.z};
          const uint32_t val[4] = {ca.y, ca.w, cb.y, cb.w};
          uint4 xv[4][C::VPL];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < C::VPL; ++v)
              xv[q][v] = *reinterpret_cast<const uint4*>(xs + (idx[q] >> C::OSH) + v * C::LPR * C::VB);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int v = 0; v < C::VPL; ++v) PFma<TX, TW, C::EPV>::run(acc + v * C::EPV, xv[q][v], val[q]);
        }
      }
    }
    if (!h.last) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[buf]);
    } else {
      // ---- epilogue of a block: de-normalise, write, squared norms ----
      const PipeLayout& P = a.L[h.prod];
      const int tile = h.work / P.nblocks, b = h.work % P.nblocks;
      const int64_t row = (int64_t)b * kRowsPerBlock + rb;
      float* yt = P.y + (size_t)tile * P.nrows * ST;
      if constexpr (PAIR) {
        // lanes 16 p + j and 16 p + 8 + j hold partial sums of the same
        // slices of both rows of pair p: each adds its partner's (one FP32
        // addition, the same value in both), then keeps in acc[0 .. 8) its
        // own row, 2 p + e = lane / 8, whose slices 8 j .. 8 j + 7 are those
        // the lane owns in the layout of the other 128-byte tiles below
#pragma unroll
        for (int i = 0; i < 2 * C::EPV; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 8);
        if ((lane >> 3) & 1) {
#pragma unroll
          for (int i = 0; i < C::EPV; ++i) acc[i] = acc[C::EPV + i];
        }
      } else if constexpr (C::SWZ) {
        // the two lanes of a row hold the same slices in swapped halves:
        // each adds the partner's partial sums of both halves
#pragma unroll
        for (int i = 0; i < C::EPV; ++i) {
          const float t0 = __shfl_xor_sync(0xffffffffu, acc[C::EPV + i], C::LPR);
          const float t1 = __shfl_xor_sync(0xffffffffu, acc[i], C::LPR);
          acc[i] += t0;
          acc[C::EPV + i] += t1;
        }
      } else if constexpr (C::ES > 1) {
        // the row's partial sums of the ES lanes (fixed order: a butterfly)
#pragma unroll
        for (int o = C::LPR; o < C::LPR * C::ES; o <<= 1)
#pragma unroll
          for (int i = 0; i < C::SPL; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
      }
      // accumulator group v holds the slices of row half hv (with the swap,
      // group 0 is the lane's own half; only that one is written and summed)
      constexpr int VOWN = C::SWZ ? 1 : C::VPL;
      const bool writer = C::SWZ || el == 0;
      float r[C::SPL];
#pragma unroll
      for (int v = 0; v < C::VPL; ++v)
#pragma unroll
        for (int e = 0; e < C::EPV; ++e) {
          const int hv = C::SWZ ? (v ^ el) : v;
          const int sl = hv * C::LPR * C::EPV + sub * C::EPV + e;
          float scale = 1.0f;
          if constexpr (C::X16)
            scale = ldexpf(1.0f, ceil_log2_exp_p(__uint_as_float(__ldg(P.in_max + tile * ST + sl))) -
                                     P.mat_scale_exp);
          else if constexpr (C::W16)
            scale = ldexpf(1.0f, -P.mat_scale_exp);
          r[v * C::EPV + e] = acc[v * C::EPV + e] * scale;
        }
      if (row < P.nrows && writer) {
#pragma unroll
        for (int v = 0; v < VOWN; ++v) {
          const int hv = C::SWZ ? (v ^ el) : v;
          float* dst = yt + (size_t)row * ST + hv * C::LPR * C::EPV + sub * C::EPV;
#pragma unroll
          for (int q = 0; q < C::EPV / 4; ++q)
            reinterpret_cast<float4*>(dst)[q] =
                make_float4(r[v * C::EPV + 4 * q], r[v * C::EPV + 4 * q + 1],
                            r[v * C::EPV + 4 * q + 2], r[v * C::EPV + 4 * q + 3]);
        }
      }
      if constexpr (C::PIXB == 16 && C::X16) {
        if (P.dot) {
          // per-slice squared norm of the block's rows, for 16-byte rows of
          // 16-bit slices: the row sums before the de-normalisation are
          // bounded (normalised inputs times 16-bit matrix values), so their
          // squares and sums are FP32 pairs (Ff), scaled by the slice's
          // power of two squared when converted to FP64.  The four lanes of
          // a row hold the same sums: each squares two of the 8 slices, the
          // sum over the warp's rows halves them between paired lanes.  The
          // warp's pairs go to this buffer's [NC][ST] area; the last warp
          // past the block end adds them in warp order and writes the
          // partials, and no warp waits for the others.  The area and its
          // counter are used again only at a block end in this buffer, after
          // a refill of the buffer, which needs every warp's release of it
          // (the last warp's after its sums).
          constexpr int DN = C::EPV / C::ES;
          Ff f[DN];
#pragma unroll
          for (int e = 0; e < C::EPV; ++e)
            if (e / DN == el) f[e % DN] = ff_square(acc[e]);
          int base = 0;
          halve_rows<DN, C::LPR * C::ES>(f, lane, base);
          constexpr int NF = halved_count(DN, C::LPR * C::ES);
          constexpr int DUP = halved_dup_mask(DN, C::LPR * C::ES);
          float2* red = dpair + (size_t)buf * C::NC * ST;
          if ((lane & DUP) == 0) {
#pragma unroll
            for (int i = 0; i < NF; ++i) red[warp * ST + el * DN + base + i] = make_float2(f[i].h, f[i].l);
          }
          __syncwarp();
          int done = 0;
          if (lane == 0) {
            __threadfence_block();
            done = atomicAdd(&dcnt[buf], 1);
            __threadfence_block();
          }
          __syncwarp();
          done = __shfl_sync(0xffffffffu, done, 0);
          if (done == C::NC - 1) {
            __threadfence_block();
            if (lane < ST) {
              Ff t = {red[lane].x, red[lane].y};
              for (int w = 1; w < C::NC; ++w) t = sum2(t, Ff{red[w * ST + lane].x, red[w * ST + lane].y});
              const int e2 =
                  2 * (ceil_log2_exp_p(__uint_as_float(__ldg(P.in_max + tile * ST + lane))) - P.mat_scale_exp);
              P.dot[(size_t)(tile * ST + lane) * P.nblocks + b] = ldexp((double)t.h + (double)t.l, e2);
            }
            __syncwarp();
            if (lane == 0) dcnt[buf] = 0;
          }
        }
      } else if (P.dot) {
        // per-slice squared norm of the block's rows: lanes sharing `sub`
        // hold the same slices (reduce over rows by shuffles), then the 16
        // consumer warps combine through shared memory in a fixed order.
        // FP64 arithmetic is slow on this part (1/64 of the FP32 rate), so
        // none of it is repeated: with lanes splitting a row's entries
        // (16-byte rows), the ES lanes of a row hold the same sums after the
        // butterfly above and each squares EPV / ES of the slices; the sum
        // over rows splits the values between paired lanes (halve_rows)
        constexpr bool SPLIT = C::ES > 1 && !C::SWZ && C::VPL == 1 && C::LPR == 1;
        constexpr int DN = SPLIT ? C::EPV / C::ES : VOWN * C::EPV;
        double d[DN];
        if constexpr (SPLIT) {
#pragma unroll
          for (int e = 0; e < C::EPV; ++e)
            if (e / DN == el) d[e % DN] = (double)r[e] * (double)r[e];
        } else {
#pragma unroll
          for (int i = 0; i < DN; ++i) d[i] = (double)r[i] * (double)r[i];
        }
        int base = 0;
        halve_rows<DN, C::LPR * C::ES>(d, lane, base);
        constexpr int NF = halved_count(DN, C::LPR * C::ES);
        constexpr int DUP = halved_dup_mask(DN, C::LPR * C::ES);
        // the staged rows of this buffer are no longer read once every
        // consumer warp is here: their area holds the [NC][ST] partials
        // (the buffer is released only after the reduction)
        double* red = reinterpret_cast<double*>(xbuf(buf));
        // consumers only, bounded: a warp that gave up earlier cannot leave
        // the others waiting
        __syncwarp();
        if (lane == 0) mbar_arrive(&redbar[0]);
        if (!mbar_wait(&redbar[0], rphase, a.wait_ns)) {
          if (lane == 0) atomicExch(a.err, 1);
          return;
        }
        if ((lane & DUP) == 0) {
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            const int j = base + i;   // index among the lane's DN squares
            int sl;
            if constexpr (SPLIT) {
              sl = el * DN + j;
            } else {
              const int v = j / C::EPV, e = j % C::EPV;
              const int hv = C::SWZ ? (v ^ el) : v;
              sl = hv * C::LPR * C::EPV + sub * C::EPV + e;
            }
            red[warp * ST + sl] = d[i];
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&redbar[1]);
        if (!mbar_wait(&redbar[1], rphase, a.wait_ns)) {
          if (lane == 0) atomicExch(a.err, 1);
          return;
        }
        rphase ^= 1u;
        if (warp == 0) {
          for (int sl = lane; sl < ST; sl += 32) {
            double t = 0.0;
            for (int w = 0; w < C::NC; ++w) t += red[w * ST + sl];
            P.dot[(size_t)(tile * ST + sl) * P.nblocks + b] = t;
          }
        }
        // order these shared-memory writes before the copies that will refill
        // the buffer once it is released
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[buf]);
    }
  }
}

size_t pipe_smem_bytes(int cap, int64_t emax, int64_t desc_bytes, int pixb, int xb, int eb, int nb,
                       uint32_t* xbytes, uint32_t* ebytes, uint32_t* dbytes) {
  const size_t x = ((size_t)(cap + 1) * pixb + 127) / 128 * 128;
  const size_t e = ((size_t)emax * eb + 127) / 128 * 128;
  const size_t d = ((size_t)desc_bytes + 127) / 128 * 128;
  if (xbytes) *xbytes = (uint32_t)x;
  if (ebytes) *ebytes = (uint32_t)e;
  if (dbytes) *dbytes = (uint32_t)d;
  // stage buffers, descriptor slots, barriers, stage identities; 16-byte
  // rows of 16-bit slices: block-end partials (8 consumer warps x 8 slices
  // of FP32 pairs per buffer) and their counters
  const size_t red = (pixb == 16 && xb == 2) ? (size_t)nb * 8 * 8 * 8 + 16 * nb : 0;
  return nb * (x + e + 256 + 128) + kDescSlots * d + 8 * (2 * nb + kDescSlots + 2) +
         16 * kDescSlots + red + 128;
}

// shared memory a pipeline CTA may use so that `minb` CTAs fit on an SM
// (228 KB per SM, 1 KB of it reserved per CTA)
constexpr size_t pipe_cta_smem_max(int minb) { return (size_t)(228 * 1024) / minb - 1024; }
// The persistent form runs with at least two CTAs per SM; narrow rows whose
// stage buffers do not fit their usual count run with as many as fit.
constexpr int kPipeMinCtas = 2;
inline int pipe_ctas_per_sm(size_t smem, int minb) {
  int c = (int)((size_t)(228 * 1024) / (smem + 1024));
  return c < minb ? c : minb;
}
constexpr int pipe_minb(int pixb) {
  return pixb >= 128 ? 2 : (pixb == 64 ? 3 : (pixb == 16 ? kPipeMinb16 : 4));
}
constexpr int pipe_nb(int pixb) { return pixb == 16 ? kPipeBufs16 : kPipeBufs; }

template <class TX, class TW, int ST, bool WIDE, bool PAIR = false>
xct_status launch_pipe(const SpmmArgs* list, int count, cudaStream_t st) {
  using C = PCfg<TX, TW, ST>;
  constexpr int EB = PAIR ? 8 : C::EB;
  // the block-end reduction reuses a buffer's staged-row area
  static_assert((size_t)C::NC * ST * sizeof(double) <= (size_t)65 * C::PIXB,
                "reduction area must fit in the staged rows of the smallest stage buffer");
  if (count < 1 || count > kMaxPipeProducts) {
    set_error("persistent product: %d products in one launch (1..%d)", count, kMaxPipeProducts);
    return XCT_ERR_UNSUPPORTED;
  }
  PipeArgs a{};
  int work = 0, cap = 0;
  int64_t emax = 0, dmax = 0;
  for (int i = 0; i < count; ++i) {
    const SpmmArgs& s = list[i];
    const Layout& L = *s.L;
    PipeLayout& P = a.L[i];
    P.blk_stage = L.blk_stage;
    P.desc = L.desc;
    P.desc_bytes = L.desc_bytes;
    P.ent = static_cast<const unsigned char*>(L.ent);
    P.nrows = L.nrows;
    P.ncols = L.ncols;
    P.cap = L.cap;
    P.nblocks = L.nblocks;
    P.ntiles = s.ntiles;
    P.work_begin = work;
    P.xs = C::X16 ? reinterpret_cast<const unsigned char*>(s.staged16)
                  : reinterpret_cast<const unsigned char*>(s.x);
    P.y = s.y;
    P.in_max = s.in_max;
    P.mat_scale_exp = s.mat_scale_exp;
    P.dot = s.dot_partial;
    work += L.nblocks * s.ntiles;
    cap = cap > L.cap ? cap : L.cap;
    if (!WIDE) emax = emax > L.emax_slots ? emax : L.emax_slots;
    dmax = dmax > L.desc_bytes ? dmax : L.desc_bytes;
  }
  a.nl = count;
  a.nwork = work;
  a.cap = cap;
  a.work = list[0].work;
  a.err = list[0].err;
  a.wait_ns = wait_limit_ns();
  static_assert(C::NB == pipe_nb(C::PIXB), "stage buffers");
  static_assert(C::PIXB != 16 || !C::X16 || (C::NC == 8 && ST == 8), "block-end partial area");
  const size_t smem = pipe_smem_bytes(cap, emax, dmax, C::PIXB, C::XB, EB, C::NB, &a.xbytes, &a.ebytes,
                                      &a.dbytes);
  static_assert(C::MINB == pipe_minb(C::PIXB), "CTAs per SM");
  const int per_sm = pipe_ctas_per_sm(smem, C::MINB);
  if (per_sm < kPipeMinCtas) {
    set_error("persistent product: %zu bytes of shared memory needed", smem);
    return XCT_ERR_UNSUPPORTED;
  }
  // the opt-in shared-memory size is a per-device attribute: set it once per
  // device and size
  static std::atomic<int> configured_for[kMaxDevices];
  int cur_dev = 0;
  XCT_TRY_CUDA(cudaGetDevice(&cur_dev));
  if (cur_dev < 0 || cur_dev >= kMaxDevices || configured_for[cur_dev].load() != (int)smem + 1) {
    XCT_TRY_CUDA(cudaFuncSetAttribute(spmm_pipe_kernel<TX, TW, ST, WIDE, PAIR>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (cur_dev >= 0 && cur_dev < kMaxDevices) configured_for[cur_dev].store((int)smem + 1);
  }
  int sms = 0;
  XCT_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur_dev));
  if (work == 0) return XCT_OK;
  const int grid = work < sms * per_sm ? work : sms * per_sm;
  XCT_TRY_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int), st));
  spmm_pipe_kernel<TX, TW, ST, WIDE, PAIR><<<grid, C::NT, smem, st>>>(a);
  count_launch();
  XCT_TRY_CUDA(cudaGetLastError());
  return XCT_OK;
}

template <class TX, class TW>
xct_status dispatch_pipe(const SpmmArgs* list, int count, cudaStream_t st) {
  // the persistent form is built for staged rows of 16, 32, 64 or 128 bytes
  // (8, 16, 32 or 64 slices in 16 bits; 4, 8, 16 or 32 in FP32)
  for (int i = 1; i < count; ++i)
    if (list[i].st != list[0].st || list[i].L->pair != list[0].L->pair) {
      set_error("persistent product: products of one launch must share the tile width and layout kind");
      return XCT_ERR_INVALID;
    }
  switch (list[0].st * PBytes<TX>::v) {
    case 128:
      if constexpr (PBytes<TX>::v == 2 && PBytes<TW>::v == 2) {
        if (list[0].L->pair) return launch_pipe<TX, TW, 64, false, true>(list, count, st);
      }
      if (list[0].L->pair) {
        set_error("persistent product: paired layouts need 16-bit slices and values");
        return XCT_ERR_INVALID;
      }
      return launch_pipe<TX, TW, 128 / PBytes<TX>::v, false>(list, count, st);
    case 64: return launch_pipe<TX, TW, 64 / PBytes<TX>::v, false>(list, count, st);
    case 32: return launch_pipe<TX, TW, 32 / PBytes<TX>::v, false>(list, count, st);
    case 16:
      if constexpr (PBytes<TX>::v == 2 && PBytes<TW>::v == 2) {
        if (list[0].L->unit == kWideRowBytes)
          return launch_pipe<TX, TW, 16 / PBytes<TX>::v, true>(list, count, st);
      }
      return launch_pipe<TX, TW, 16 / PBytes<TX>::v, false>(list, count, st);
    default:
      set_error("persistent product: unsupported tile width %d", list[0].st);
      return XCT_ERR_UNSUPPORTED;
  }
}

xct_status pipe_any(const SpmmArgs* list, int count, cudaStream_t s) {
  const xct_dtype t = list[0].storage;
  for (int i = 1; i < count; ++i)
    if (list[i].storage != t) {
      set_error("persistent product: products of one launch must share the storage type");
      return XCT_ERR_INVALID;
    }
  switch (t) {
    case XCT_F32: return dispatch_pipe<float, float>(list, count, s);
    case XCT_F16: return dispatch_pipe<__half, __half>(list, count, s);
    case XCT_BF16: return dispatch_pipe<__nv_bfloat16, __nv_bfloat16>(list, count, s);
    case XCT_F16A: return dispatch_pipe<float, __half>(list, count, s);
    case XCT_BF16A: return dispatch_pipe<float, __nv_bfloat16>(list, count, s);
    default:
      set_error("persistent product: unknown storage type");
      return XCT_ERR_INVALID;
  }
}

}  // namespace

// The persistent form needs 16-byte lane vectors, staged rows of 16, 32, 64
// or 128 bytes and two buffers in the shared memory of one of its CTAs.
bool spmm_pipe_applies(const SpmmArgs& a) {
  const int pixb = a.st * (stages16(a.storage) ? 2 : 4);
  if ((pixb != 128 && pixb != 64 && pixb != 32 && pixb != 16) || !a.work || !a.err) return false;
  if (a.L->nblocks == 0) return false;
  if (a.L->unit != kEntryRowBytes && (pixb != a.L->unit || !stages16(a.storage))) return false;
  const int64_t emax = a.L->unit == kEntryRowBytes ? a.L->emax_slots : 0;   // wide: not staged
  if (a.L->pair && (pixb != kEntryRowBytes || !stages16(a.storage))) return false;
  return pipe_smem_bytes(a.L->cap, emax, a.L->desc_bytes, pixb, stages16(a.storage) ? 2 : 4,
                         a.L->ebytes,
                         pipe_nb(pixb), nullptr, nullptr, nullptr) <= pipe_cta_smem_max(kPipeMinCtas);
}

xct_status spmm_pipe(const SpmmArgs& a, cudaStream_t s) { return pipe_any(&a, 1, s); }

bool spmm_pipe_multi_applies(const SpmmArgs* list0, int count) {
  if (count < 1 || count > kMaxPipeProducts) return false;
  SpmmArgs list[kMaxPipeProducts];
  for (int i = 0; i < count; ++i) list[i] = on_product_layout(list0[i]);
  int cap = 0;
  int64_t emax = 0, dmax = 0;
  for (int i = 0; i < count; ++i) {
    if (!spmm_pipe_applies(list[i]) || list[i].storage != list[0].storage ||
        list[i].st != list[0].st || list[i].L->unit != list[0].L->unit ||
        list[i].L->pair != list[0].L->pair)
      return false;
    cap = cap > list[i].L->cap ? cap : list[i].L->cap;
    if (list[i].L->unit == kEntryRowBytes)
      emax = emax > list[i].L->emax_slots ? emax : list[i].L->emax_slots;
    dmax = dmax > list[i].L->desc_bytes ? dmax : list[i].L->desc_bytes;
  }
  const int pixb = list[0].st * (stages16(list[0].storage) ? 2 : 4);
  return pipe_smem_bytes(cap, emax, dmax, pixb, stages16(list[0].storage) ? 2 : 4,
                         list[0].L->ebytes, pipe_nb(pixb),
                         nullptr, nullptr, nullptr) <= pipe_cta_smem_max(kPipeMinCtas);
}

xct_status spmm_pipe_multi(const SpmmArgs* list0, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxPipeProducts) {
    set_error("persistent product: %d products in one launch (1..%d)", count, kMaxPipeProducts);
    return XCT_ERR_UNSUPPORTED;
  }
  SpmmArgs list[kMaxPipeProducts];
  for (int i = 0; i < count; ++i) list[i] = on_product_layout(list0[i]);
  return pipe_any(list, count, s);
}

}  // namespace xct

// Internal declarations of libxct.so (not part of the C-ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "xct.h"

namespace xct {

// ---------------------------------------------------------------------------
// errors, allocation, launch accounting
// ---------------------------------------------------------------------------

void set_error(const char* fmt, ...);
// limit of the bounded waits inside the persistent kernels (xct_set_wait_limit)
uint64_t wait_limit_ns();
constexpr int kMaxDevices = 64;   // per-device caches of launch attributes
extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Device allocation through the configured allocator (cudaMallocAsync by
// default).  Returns nullptr and sets the error message on failure.
void* dalloc(size_t bytes, cudaStream_t s);
void dfree(void* p, size_t bytes, cudaStream_t s);

// An NVTX range for the duration of an entry point (a no-op unless a
// profiler is attached), so traces show the library's calls by name.
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

// The fixed working array of xct_project_noalloc (noalloc.cu): resolve its
// device address on `device` (made current for the call, then restored), so
// that the array is resident there before the first call that relies on it.
xct_status noalloc_reserve(int device);

#define XCT_TRY_CUDA(call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ::xct::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                       __FILE__, __LINE__);                                  \
      return XCT_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

#define XCT_TRY(expr)                  \
  do {                                 \
    xct_status st_ = (expr);           \
    if (st_ != XCT_OK) return st_;     \
  } while (0)

// A set of device allocations released together (in reverse order).
struct Arena {
  struct Item { void* p; size_t n; };
  std::vector<Item> items;
  cudaStream_t stream = nullptr;
  explicit Arena(cudaStream_t s = nullptr) : stream(s) {}
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() { release(); }
  template <class T>
  xct_status get(T** out, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 256;
    void* p = dalloc(bytes, stream);
    if (!p) { *out = nullptr; return XCT_ERR_OOM; }
    items.push_back({p, bytes});
    *out = static_cast<T*>(p);
    return XCT_OK;
  }
  void release() {
    for (size_t i = items.size(); i-- > 0;) dfree(items[i].p, items[i].n, stream);
    items.clear();
  }
  // hand ownership of all items to another arena
  void move_to(Arena& other) {
    for (auto& it : items) other.items.push_back(it);
    items.clear();
  }
};

// storage forms: 16-bit matrix values; 16-bit (normalised) staged slices;
// binary16 (rather than bfloat16) values
inline bool matrix16(xct_dtype t) { return t != XCT_F32; }
inline bool stages16(xct_dtype t) { return t == XCT_F16 || t == XCT_BF16; }
inline bool half_values(xct_dtype t) { return t == XCT_F16 || t == XCT_F16A; }
inline bool valid_storage(int t) { return t >= XCT_F32 && t <= XCT_BF16A; }

// ---------------------------------------------------------------------------
// kernel layout of one matrix (A or A^T)
// ---------------------------------------------------------------------------

constexpr int kRowsPerBlock = 64;              // rows of one thread block
constexpr int kQuads = kRowsPerBlock / 4;      // 4-row groups per block

// Packed entries name their staged row by its byte offset at 128 bytes per
// row (position * 128): a tile with PIXB-byte staged rows finds the row at
// offset >> log2(128 / PIXB), one shift-add per entry.  16-bit entries hold
// {value bits (low 16), offset (high 16)}, FP32 entries {offset (low 32),
// value bits (high 32)}.  The offset of the zero slot (position cap) must fit
// in 16 bits.
constexpr int kEntryRowBytes = 128;
constexpr int kMaxStageCap = 65535 / kEntryRowBytes - 1;
// wide-stage layouts for few slices: 16-byte rows addressed at 16 bytes per
// row (up to 4094 rows a stage), entries streamed from global memory by the
// consumers instead of staged
constexpr int kWideRowBytes = 16;
// stage capacities (rows) of the wide layouts of A and A^T: 1524 rows of A
// (24 KB, four CTAs still fit an SM) measured 5% faster projections than
// 1016; for A^T 1016 measured best (762 and 1270 slower)
constexpr int kWideCapA = 1524;
constexpr int kWideCapAT = 1016;
constexpr int kWideGap = 16;
// log2(128 / pixb) for staged rows of pixb = 2 .. 128 bytes
__host__ __device__ constexpr int entry_shift(int pixb) {
  return pixb >= 128 ? 0 : pixb == 64 ? 1 : pixb == 32 ? 2 : pixb == 16 ? 3 : pixb == 8 ? 4
       : pixb == 4 ? 5 : 6;
}

// One (stage, quad) segment: the entries of 4 consecutive rows interleaved in
// chunks of 4 entries; `off` counts entries from the start of `ent`.
struct __align__(16) Seg {
  int64_t off;
  uint16_t cnt[4];
};

// A stage descriptor: what the persistent product's producer needs about
// one stage, stored at a fixed stride so that its address follows from the
// stage index alone and one bulk copy, requested several stages ahead, brings
// it in: the head, the stage's kQuads segment headers, then its run list
// padded to the layout's longest one with closing pairs.
struct __align__(16) StageDescHead {
  int64_t e0;          // first packed slot of the stage
  uint32_t slots;      // packed slots of the stage
  uint16_t np;         // staged rows
  uint16_t nr;         // run-list pairs (even)
};
inline int64_t stage_desc_bytes(int64_t run_stride) {
  return (int64_t)sizeof(StageDescHead) + kQuads * 16 + 8 * run_stride;
}

struct Layout {
  int64_t nrows = 0, ncols = 0;
  int32_t nblocks = 0;
  int32_t cap = 0;             // staged vectors per stage (the zero slot is `cap`)
  int32_t ebytes = 0;          // 4: {u16 index, 16-bit value}; 8: {u32 index, f32}
  int64_t nstages = 0;
  int64_t nslots = 0;          // stored entries including padding
  int64_t footprint = 0;       // staged vectors over all stages
  int64_t* blk_stage = nullptr;   // [nblocks + 1] stage ranges of the blocks
  int64_t* stage_pix = nullptr;   // [nstages + 1] offsets into pix
  int32_t* stage_np = nullptr;    // [nstages] staged rows of each stage
  int32_t* pix = nullptr;         // staged input row ids, stage by stage
  Seg* seg = nullptr;             // [nstages * kQuads]
  void* ent = nullptr;            // packed entries
  int64_t* stage_ent = nullptr;   // [nstages + 1] first slot of each stage's entries
  int64_t emax_slots = 0;         // largest stage, in slots
  // contiguous runs of each stage's staged rows (see run_fill_kernel)
  int64_t* stage_run = nullptr;   // [nstages + 1] offsets into runs (even)
  int2* runs = nullptr;           // (first row id, first position) pairs
  int64_t nruns = 0;              // pairs over all stages
  int64_t run_max = 0;            // largest stage list, in pairs
  unsigned char* desc = nullptr;  // [nstages] stage descriptors of desc_bytes each
  int64_t desc_bytes = 0;
  // bytes per staged row in the entries' offsets (kEntryRowBytes, or 16 for
  // a wide-stage layout whose offsets address 16-byte rows directly)
  int32_t unit = kEntryRowBytes;
  // the wide-stage layout of the same matrix for 16-byte staged rows (built
  // with XCT_PLAN_FEW_SLICES), used in place of this one for such tiles
  const Layout* wide = nullptr;
  // the paired layout of the same matrix for 128-byte rows of 16-bit slices
  // (built with XCT_PLAN_PAIRED_ROWS), used in place of this one for such
  // tiles; `pair` marks a paired layout itself (its stages, staged rows and
  // runs are those of the plain layout, its segments and 8-byte slots its own)
  const Layout* paired = nullptr;
  bool pair = false;
  int64_t gathers = 0;         // paired: distinct columns of the pairs over all stages
                               // (the staged-row reads of one tile, padding aside)
  int64_t bytes = 0;
};

// Paired layout (XCT_PLAN_PAIRED_ROWS).  Rows 2p and 2p + 1 of a quad form
// pair p.  A pair's entries in a stage are split into shared slots, one per
// column both rows cross ({offset << 16 | value of row 2p, offset << 16 |
// value of row 2p + 1}), and split slots, one column of each row ({offset0 <<
// 16 | value0, offset1 << 16 | value1}, the zero slot with value 0 where one
// row has no entry left).  Two lanes of a pair take alternate slots (a chunk
// is 2 slots).  A (stage, quad) segment holds the shared region, then the
// split region; each region is a sequence of groups of kPairUA (shared) or
// kPairUB (split) chunks, and in a group the kPair* slots of each (pair, lane)
// are contiguous: slot u of lane e of pair p in group g of the shared region
// lies at g * 4 * kPairUA + (2 p + e) * kPairUA + u.  Seg::cnt holds the
// chunk counts {shared of pair 0, split of pair 0, shared of pair 1, split
// of pair 1}; each region has as many groups as its longer pair needs.
constexpr int kPairUA = 4;
constexpr int kPairUB = 2;

// Shared memory of one pipeline buffer (staged rows of `pixb` bytes, the
// stage's packed entries, its segment headers and header) with its share of
// the stage-descriptor slots (four slots over two buffers) -- see
// spmm_pipe.cu.
inline size_t pipe_buffer_bytes(const Layout& L, int pixb) {
  size_t x = ((size_t)(L.cap + 1) * pixb + 127) / 128 * 128;
  size_t e = ((size_t)L.emax_slots * L.ebytes + 127) / 128 * 128;
  size_t d = ((size_t)L.desc_bytes + 127) / 128 * 128;
  return x + e + 2 * d + 128 * 2 + 256;
}
#ifndef XCT_PIPE_BUFS
#define XCT_PIPE_BUFS 2
#endif
// stage buffers of a pipeline CTA (the producer fills up to kPipeBufs - 1
// stages ahead of the consumers)
constexpr int kPipeBufs = XCT_PIPE_BUFS;
static_assert(kPipeBufs == 2 || kPipeBufs == 3, "pipeline buffers");
// stage buffers and CTAs per SM of the pipeline with 16-byte staged rows
#ifndef XCT_PIPE_BUFS16
#define XCT_PIPE_BUFS16 2
#endif
#ifndef XCT_PIPE_MINB16
#define XCT_PIPE_MINB16 4
#endif
constexpr int kPipeBufs16 = XCT_PIPE_BUFS16;
constexpr int kPipeMinb16 = XCT_PIPE_MINB16;
// shared memory one pipeline CTA with 128-byte staged rows may use for its
// buffers (two such CTAs share an SM; the rest of a CTA's 113 KB goes to the
// barriers and run lists)
constexpr size_t kPipeSmemLimit = 110 * 1024;
// first stage capacity tried for each entry size (reduced until the buffers
// fit in kPipeSmemLimit)
constexpr int kPipeCap16 = kPipeBufs == 2 ? 280 : 184;
constexpr int kPipeCap32 = kPipeBufs == 2 ? 200 : 132;

struct Plan {
  xct_geometry g{};
  std::vector<double> cs;       // host angle table [M][2]
  xct_dtype storage = XCT_F32;
  uint32_t flags = 0;
  int device = 0;
  int64_t nray = 0, npix = 0, nnz = 0;
  int32_t* pix_order = nullptr;  // natural pixel -> ordered id
  int32_t* pix_inv = nullptr;    // ordered id -> natural pixel
  int32_t* ray_order = nullptr;
  int32_t* ray_inv = nullptr;
  Layout la, lat;
  Layout law, latw;              // wide-stage layouts (XCT_PLAN_FEW_SLICES)
  Layout lap, latp;              // paired layouts (XCT_PLAN_PAIRED_ROWS)
  int32_t mat_scale_exp = 0;     // k: stored value = RN(l * 2^k)
  int* err = nullptr;            // device flag: a bounded wait in a kernel ran out
  // kept FP64 matrices (ordered ids), only with XCT_PLAN_KEEP_F64
  int64_t* a_rowptr = nullptr; int32_t* a_col = nullptr; double* a_val = nullptr;
  int64_t* t_rowptr = nullptr; int32_t* t_col = nullptr; double* t_val = nullptr;
  Arena mem;                     // everything above lives here
  xct_stats stats{};
  std::map<int, int> tile_choice;  // measured slice-tile width per slice count
};

// plan building (plan.cu)
xct_status build_plan(Plan& p, cudaStream_t s);
// y = A x without the stored matrix: every ray traced again (plan.cu)
xct_status matfree_project(const Plan& p, const double* cs_dev, const float* x, float* y, int S,
                           cudaStream_t s);
// x = A^T y without the stored matrix: pixel-driven, lengths from each
// pixel's boundary planes, equal to the stored values (plan.cu)
xct_status matfree_backproject(const Plan& p, const double* cs_dev, const float* y, float* x, int S,
                               cudaStream_t s);
// the double-precision form (f64.cu): products and CGLS on the kept FP64
// matrices, natural-layout device vectors; f64_cgls writes log [iters+1][S][2]
// (device, nullable) and whether any slice was active after the start
xct_status f64_apply(Plan& p, bool transposed, const double* in, double* out, int S,
                     cudaStream_t s);
xct_status f64_cgls(Plan& p, const double* y, double* x, int S, int iters, bool x0, double* log,
                    int* any_active, cudaStream_t s);
xct_status export_matrix(Plan& p, int what, int64_t* rowptr, int32_t* col,
                         double* val, int64_t* nnz);

// device exclusive scans (scan.cu): out[i] = sum_{j<i} in[j], out[n] = total
xct_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
xct_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// products (spmm.cu) on the internal vector layout [tile][rows][st] float32
// ---------------------------------------------------------------------------

struct SpmmArgs {
  const Layout* L;
  const float* x;          // input [ntiles][L->ncols][st]
  float* y;                // output [ntiles][L->nrows][st]
  int st;                  // slices per tile
  int ntiles;
  xct_dtype storage;
  int mat_scale_exp;
  const uint32_t* in_max;  // per slice max |x| bits (16-bit storage) [ntiles*st]
  double* dot_partial;     // nullable: [ntiles*st][nblocks] sum of y^2 per block
  uint16_t* staged16;      // 16-bit storage: scratch [ntiles][L->ncols][st] for the
                           // normalised 16-bit copy of x (unused for FP32)
  int* work;               // scratch: one work counter (persistent form)
  int* err;                // device flag set to 1 if a bounded wait ran out
};
// The layout a product runs on: the matrix's wide-stage layout, where the
// plan built one, for 16-byte staged rows of 16-bit slices; its paired
// layout, where the plan built one, for 128-byte staged rows of 16-bit
// slices; else its own.
inline SpmmArgs on_product_layout(SpmmArgs a) {
  if (a.L->wide && stages16(a.storage) && a.st * 2 == kWideRowBytes) a.L = a.L->wide;
  else if (a.L->paired && stages16(a.storage) && a.st * 2 == kEntryRowBytes) a.L = a.L->paired;
  return a;
}
xct_status spmm(const SpmmArgs& a, cudaStream_t s);   // = spmm_stage + spmm_run
// 16-bit storage: the normalised 16-bit copy of the input (no-op for FP32)
xct_status spmm_stage(const SpmmArgs& a, cudaStream_t s);
// the product kernel itself
xct_status spmm_run(const SpmmArgs& a, cudaStream_t s);
// the persistent warp-specialised form (spmm_pipe.cu); false if it does not
// apply to this layout / tile width (the caller then uses the staged form)
bool spmm_pipe_applies(const SpmmArgs& a);
xct_status spmm_pipe(const SpmmArgs& a, cudaStream_t s);
// several products (same storage type, 128-byte rows) in one persistent
// launch sharing one work counter (list[0].work) -- the batched solver
constexpr int kMaxPipeProducts = 8;
bool spmm_pipe_multi_applies(const SpmmArgs* list, int count);
xct_status spmm_pipe_multi(const SpmmArgs* list, int count, cudaStream_t s);
// number of per-slice partial sums spmm() writes for dot_partial (per slice):
// one per block of rows
int spmm_dot_count(const SpmmArgs& a);
bool spmm_supported(xct_dtype storage, int st);
int pick_slices_per_tile(xct_dtype storage, int S);

// regularisation (tv.cu)
xct_status tv_launch(const float* x, int n, int S, double eps, double weight, float* grad,
                     bool accumulate, double* partial, double* value_dev, cudaStream_t s);
int tv_partials(int n);
xct_status adam_launch(float* x, const float* g, float* m, float* v, int64_t count, double lr,
                       double beta1, double beta2, double eps, int step, cudaStream_t s);

// vector kernels (vec.cu)
xct_status to_internal(const float* nat, float* in, const int32_t* inv_order,
                       int64_t rows, int S, int st, int ntiles, uint32_t* max_bits,
                       cudaStream_t s);
xct_status to_natural(const float* in, float* nat, const int32_t* inv_order,
                      int64_t rows, int S, int st, int ntiles, cudaStream_t s);

}  // namespace xct

// The opaque handle of the C-ABI is the plan itself.
struct xct_plan_s : public xct::Plan {};

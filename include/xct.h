/*
 * xct.h -- C-ABI of libxct.so: a GB300 (sm_103a) memoized parallel-beam
 * projector (Siddon system matrix A and its explicit transpose, applied to
 * batches of slices that share them) and a device-resident CGLS solver.
 *
 * Method: "Petascale XCT: 3D Image Reconstruction with Hierarchical
 * Communications on Multi-GPU Nodes" (SC20).  Section / equation references
 * below are to that paper.
 *
 * Conventions for every entry point:
 *   - Status codes only: no abort, no exception crosses the ABI.  On an error
 *     xct_last_error() returns a thread-local message.  Arguments are checked
 *     before any GPU work is queued.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream are stream-ordered and return before the GPU work is
 *     done, except where stated.
 *   - Vector arguments (images x, sinograms y) may be device pointers or host
 *     pointers (pageable or pinned); the library detects which.  Host
 *     arguments are copied in and out inside the call, which then
 *     synchronises `stream` before returning.  xct_project and
 *     xct_backproject with host vectors and more slices than one slice tile
 *     pipeline the copies per tile on two internal copy streams (one per
 *     direction) so they overlap the other tiles' products; pinned host
 *     memory lets them run concurrently.
 *   - The caller owns every x / y buffer.  A plan owns its matrices; they are
 *     released by xct_free().
 *   - Image layout: x[s][iy][ix], S slices of n*n float32, slice-major,
 *     natural pixel order.  Sinogram layout: y[s][k][j], S slices of
 *     n_angles*n_det float32.
 *
 * Geometry (Sec. II-A, parallel beam; conventions fixed by this library):
 *   pixel (ix, iy) covers [ix - n/2, ix - n/2 + 1] x [iy - n/2, iy - n/2 + 1];
 *   ray (k, j) is the line {P : P . (cos th_k, sin th_k) = t_j},
 *   t_j = (j - (n_det - 1)/2) * det_spacing + det_offset, traversed along
 *   (-sin th_k, cos th_k).  A[ray, pixel] = length of the ray in the pixel
 *   (Siddon's method, FP64, segments shorter than min_seg dropped).
 */
#ifndef XCT_H
#define XCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XCT_OK = 0,
  XCT_ERR_INVALID = 1,      /* bad argument or geometry */
  XCT_ERR_OOM = 2,          /* an allocation failed (nothing leaked) */
  XCT_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  XCT_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
  XCT_ERR_BREAKDOWN = 5,    /* CGLS: every slice stopped at k = 0 (zero data) */
  XCT_ERR_UNSUPPORTED = 6   /* valid request the library does not handle */
} xct_status;

/* Storage precision of a plan (Sec. III-C).  XCT_F32: values and staged
 * vectors in float32.  XCT_F16 / XCT_BF16: matrix values stored as
 * RN16(l * 2^k) (k = 15 for binary16, 0 for bfloat16), input vectors
 * normalised per slice by 2^-ceil(log2 max|v_s|) and staged in 16 bits,
 * products accumulated in float32, outputs float32.  XCT_F16A / XCT_BF16A:
 * the same 16-bit matrix values with the input vectors staged in float32
 * (no normalisation): the matrix bytes of the 16-bit forms, the vector
 * rounding of the float32 form. */
typedef enum {
  XCT_F32 = 0,
  XCT_F16 = 1,
  XCT_BF16 = 2,
  XCT_F16A = 3,
  XCT_BF16A = 4
} xct_dtype;

typedef struct {
  int32_t n;              /* grid side (pixels), 1 <= n <= 32768 */
  int32_t n_angles;       /* M >= 1 */
  int32_t n_det;          /* N_d >= 1; n_angles * n_det < 2^31 */
  int32_t hilbert_tile;   /* T of the T x T tiles of Sec. III-A1; 0 -> 8 */
  const double* cos_sin;  /* host [n_angles][2] (cos, sin) or NULL for
                             th_k = k*pi/n_angles via the host C library;
                             copied by xct_plan */
  double det_spacing;     /* detector bin spacing, finite, != 0 (1.0) */
  double det_offset;      /* detector offset, finite (0.0) */
  double min_seg;         /* drop segments shorter than this, >= 0 (1e-9) */
} xct_geometry;

typedef struct xct_plan_s* xct_plan_t;

/* Plan flags. */
#define XCT_PLAN_KEEP_F64 1u  /* keep the FP64 CSR of A and A^T on the device
                                 for xct_plan_export (12 bytes per entry each) */
#define XCT_PLAN_AUTOTUNE 2u  /* choose each matrix's stage capacity -- the
                                 pixels (of A) or rays (of A^T) a CTA stages at
                                 a time -- by timing its product on the widest
                                 slice tile (about 3x the layout time) */
#define XCT_PLAN_FEW_SLICES 4u  /* XCT_F16 / XCT_BF16 only: also build
                                   wide-stage layouts of A and A^T (stages of
                                   up to 1524 (A) / 1016 (A^T) staged rows,
                                   the packed entries read straight from
                                   device memory) for
                                   products of at most 8 slices, where the
                                   matrix stream from HBM is the lowest roof
                                   (Sec. III-B, roofline: input buffering of
                                   many columns per stage); about doubles the
                                   plan's memory and build time */
#define XCT_PLAN_NARROW_TILES 8u  /* 16-bit matrix storage only: order the
                                     entries of each 4-row group so that
                                     16- and 32-slice tiles (32- and 64-byte
                                     staged rows) read rows in distinct
                                     shared-memory bank groups (measured 7.7%
                                     / 2.7% faster products; 64-slice tiles
                                     0.7% slower, 8-slice tiles of a plan
                                     without XCT_PLAN_FEW_SLICES 3% slower) */
#define XCT_PLAN_PAIRED_ROWS 16u  /* XCT_F16 / XCT_BF16 only: also build
                                     paired layouts of A and A^T for 64-slice
                                     tiles (128-byte staged rows): the two
                                     rows of each pair (neighbouring angles
                                     through one bin; neighbouring pixels)
                                     share one gather of a staged row for
                                     every column both cross (Sec. III-B
                                     register reuse, taken across rows), so
                                     a product reads 0.71 (A) / 0.75 (A^T)
                                     of the staged rows it otherwise would
                                     at 512^2 x 768 angles (0.86 / 0.75 at
                                     1536^2 x 1024, where neighbouring
                                     angles diverge more; the 64-slice
                                     CGLS of 512^2 x 768 x 512 measured 5%
                                     faster); products of other tile widths
                                     use the plan's own layouts, and so do
                                     64-slice tiles if the paired layouts'
                                     stage buffers do not fit the product
                                     kernel (they are then not kept).  Adds
                                     about 1.2x the packed entries of A and
                                     A^T to the plan (8 bytes a slot) */

/*
 * xct_plan -- build the memoized operator (Sec. II-B memoization; Sec. III-A1
 * Hilbert ordering; Sec. III-B input buffering; Sec. III-C storage).
 * Traces every ray on the GPU (count pass, scan, fill pass), orders pixels
 * and rays along the pseudo-Hilbert curve, forms the explicit transpose
 * (stable in ray order), and packs both into the staged kernel layout.
 * Synchronous: returns when the plan is ready (the work runs on `stream`).
 * `out` receives the plan; on error *out is NULL and nothing is leaked.
 */
xct_status xct_plan(const xct_geometry* g, xct_dtype storage, uint32_t flags,
                    void* stream, xct_plan_t* out);

/* Release a plan and everything it owns (NULL is a no-op).  Synchronises
 * the device work of the plan first. */
void xct_free(xct_plan_t plan);

/*
 * xct_project -- y = A x for S slices sharing A (Sec. II-B: the rays u_{*,j}
 * trace the same voxels in every slice; Sec. III-B2: fused A X = B).
 * x: [S][n][n] float32, y: [S][n_angles][n_det] float32 (overwritten).
 * S = 0 is a no-op.  Arithmetic per the plan's storage precision.
 */
xct_status xct_project(xct_plan_t plan, const float* x, float* y, int32_t S,
                       void* stream);

/*
 * xct_backproject -- x = A^T y with the stored transpose (Sec. III-B: the
 * same kernel serves projection and back projection).  y: [S][M][N_d],
 * x: [S][n][n] (overwritten).  Exact adjoint of xct_project in F32 storage.
 */
xct_status xct_backproject(xct_plan_t plan, const float* y, float* x,
                           int32_t S, void* stream);

/*
 * xct_project_matfree -- y = A x without the stored matrix: every ray is
 * traced again on the GPU with the plan's geometry and arithmetic (the
 * recomputation that memoizing A avoids, Sec. II-B) and RN32(length) * x is
 * accumulated in FP32, 8 slices per trace.  A comparison point and the form
 * for grids whose A does not fit in memory.  x, y: natural layouts, host or
 * device.  Synchronous.
 */
xct_status xct_project_matfree(xct_plan_t plan, const float* x, float* y, int32_t S,
                               void* stream);

/*
 * xct_backproject_matfree -- x = A^T y without the stored matrix, pixel by
 * pixel: for each pixel and angle, the few rays whose line can meet the
 * pixel are tested, and a ray's length in the pixel is taken from its
 * crossings of the pixel's four boundary planes with the plan's FP64
 * arithmetic -- the segment the trace of xct_plan keeps, so the lengths
 * equal the stored FP64 values bit for bit (for min_seg > 0; with
 * min_seg = 0 the trace also keeps slivers below 1e-14 left by rounding
 * where two crossings coincide, which this rule does not).  RN32(length) * y is summed in
 * FP32 over ascending ray ids, 8 slices per pass.  The transpose of
 * xct_project_matfree; with it, CGLS needs no stored matrix (Sec. II-B's
 * alternative to memoization).  y, x: natural layouts, host or device.
 * Synchronous.
 */
xct_status xct_backproject_matfree(xct_plan_t plan, const float* y, float* x, int32_t S,
                                   void* stream);

/*
 * xct_cgls_matfree -- xct_cgls with the matrix-free products above (no
 * stored matrix is read): the same recurrence, FP32 vectors and FP64
 * per-slice scalars, the same stop and XCT_ERR_BREAKDOWN rules, resid as
 * there; flags: XCT_CGLS_X0 only.  Each product traces the geometry again,
 * so a solve costs hundreds of times the memoized one (Sec. II-B); it is
 * the form for grids whose matrix does not fit.  Synchronous.
 */
xct_status xct_cgls_matfree(xct_plan_t plan, const float* y, float* x, int32_t S,
                            int32_t iters, uint32_t flags, double* resid, void* stream);

/*
 * xct_project_f64 / xct_backproject_f64 / xct_cgls_f64 -- the double-precision
 * form that Sec. V measures the single, half and mixed forms against: the
 * plan's kept FP64 matrix values (the plan must be built with
 * XCT_PLAN_KEEP_F64, else XCT_ERR_INVALID), float64 vectors, FP64 FMAs and
 * FP64 CGLS scalars.  x: [S][n][n] float64, y: [S][n_angles][n_det] float64
 * (natural layouts as above), host or device.  xct_cgls_f64 runs the
 * recurrence of xct_cgls (flags: XCT_CGLS_X0 only; resid as there; the same
 * stop and XCT_ERR_BREAKDOWN rules) with launches issued directly (no
 * graph), and returns when the solve is done.  The products are bound by
 * the GPU's FP64 FMA rate.
 */
xct_status xct_project_f64(xct_plan_t plan, const double* x, double* y, int32_t S,
                           void* stream);
xct_status xct_backproject_f64(xct_plan_t plan, const double* y, double* x, int32_t S,
                               void* stream);

/* CGLS flags. */
#define XCT_CGLS_X0 1u        /* start from the x passed in (else from 0) */
#define XCT_CGLS_NO_GRAPH 2u  /* launch kernels directly, no CUDA graph */
#define XCT_CGLS_TIMING 4u    /* time each phase with CUDA events (implies
                                 NO_GRAPH); read back with xct_plan_stats */

/*
 * xct_cgls -- least squares min ||y_s - A x_s|| for each slice s (Eq. 1 with
 * R = 0 and no constraint), `iters` CGLS iterations: one initial back
 * projection, then one projection and one back projection per iteration
 * (Table IV footnote: 30 projections, 31 back projections).  Dot products,
 * norms and the alpha/beta updates run on the GPU in FP64, per slice.
 * y: [S][M][N_d] float32; x: [S][n][n] float32, in = x0 if XCT_CGLS_X0,
 * out = solution.  resid: NULL, or host/device double [iters+1][S][2]
 * receiving (||r_k||, ||A^T r_k||) per iteration and slice.
 * A slice whose gamma or delta becomes exactly 0 stops silently (its x is
 * final).  Returns XCT_ERR_BREAKDOWN only if every slice stopped at k = 0;
 * x then holds x0 (or zeros).  The iteration runs as one CUDA graph unless
 * flags say otherwise.
 */
xct_status xct_cgls(xct_plan_t plan, const float* y, float* x, int32_t S,
                    int32_t iters, uint32_t flags, double* resid, void* stream);
xct_status xct_cgls_f64(xct_plan_t plan, const double* y, double* x, int32_t S,
                        int32_t iters, uint32_t flags, double* resid, void* stream);

/* CGLS state flags (xct_cgls_state). */
#define XCT_CGLS_SAVE 32u    /* write the state after the last iteration */
#define XCT_CGLS_RESUME 64u  /* start from the state instead of x0 / zero */

/*
 * xct_cgls_state -- xct_cgls with an exact checkpoint: with XCT_CGLS_SAVE
 * the state after the last iteration (per slice x, r, p in natural layouts,
 * the FP64 gamma = ||A^T r||^2 and the stop flag, and the iteration count)
 * is written to `state`; with XCT_CGLS_RESUME the solve starts from it (y
 * and x0 are not read) and continues exactly as the uninterrupted solve
 * would: k iterations, save, then m iterations from the state give the x
 * and residual log of k + m iterations bit for bit (same plan and S).  Both
 * flags may be set (continue and save again).  state: host or device,
 * xct_cgls_state_bytes(plan, S) bytes, owned by the caller; resid[0] of a
 * resumed solve is the saved iteration's entry.  XCT_ERR_INVALID for a
 * state of another plan or slice count.  The paper has no counterpart.
 */
int64_t xct_cgls_state_bytes(xct_plan_t plan, int32_t S);
xct_status xct_cgls_state(xct_plan_t plan, const float* y, float* x, int32_t S, int32_t iters,
                          uint32_t flags, double* resid, void* state, void* stream);

/*
 * xct_tv -- smoothed total variation, the regulariser R(x) of Eq. 1 as this
 * library reads it: TV_eps(x_s) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2) per
 * slice with forward differences dx = x[i][j+1] - x[i][j], dy = x[i+1][j] -
 * x[i][j] (0 past the last column / row).  One fused pass computes the value
 * and the gradient.  x: device [S][n][n] float32.  grad: device [S][n][n]
 * (overwritten with weight * dTV/dx) or NULL.  value: NULL or host/device
 * double [S] receiving weight * TV_eps(x_s) (a host pointer makes the call
 * synchronous).  eps > 0.
 */
xct_status xct_tv(const float* x, int32_t n, int32_t S, double eps, double weight,
                  float* grad, double* value, void* stream);

/*
 * xct_adam -- one Adam step on `count` float32 parameters in place (the
 * update of the gradient iteration of Sec. II-A for the regularised cost of
 * Eq. 1): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * x -= lr / (1 - b1^step) * m / (sqrt(v) / sqrt(1 - b2^step) + eps).
 * x, g, m, v: device pointers; step >= 1 counts from 1.
 */
xct_status xct_adam(float* x, const float* g, float* m, float* v, int64_t count, double lr,
                    double beta1, double beta2, double eps, int32_t step, void* stream);

/*
 * xct_tv_reconstruct -- the regularised reconstruction of Eq. 1 with
 * R(x) = lam * TV_eps(x): `steps` Adam steps (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8) on 0.5 ||y_s - A x_s||^2 + lam TV_eps(x_s), summed over slices.
 * Each step projects, forms the residual, back projects it (the data-fit
 * gradient), adds lam * grad TV_eps and updates x, all on the GPU.
 * y: [S][M][N_d], x: [S][n][n] (in: start if flags & 1, else zeros; out:
 * result), host or device.  loss: NULL or host/device double [steps] with the
 * cost at each step before its update.  Synchronous.
 */
xct_status xct_tv_reconstruct(xct_plan_t plan, const float* y, float* x, int32_t S,
                              int32_t steps, double lr, double lam, double eps, uint32_t flags,
                              double* loss, void* stream);

/*
 * xct_datafit -- the data term of Eq. 1 and its residual: r = q - y and
 * value = sum over slices of 0.5 ||r_s||^2 (FP64, summed in a fixed order),
 * for q = A x computed by xct_project; the gradient of the data term is then
 * xct_backproject(r).  q, y, r: device float32 [S][len], r not overlapping q or y;
 * value: NULL, or a host (the call is then synchronous) or device double.
 * XCT_ERR_INVALID for host vectors or negative sizes.
 */
xct_status xct_datafit(const float* q, const float* y, float* r, int64_t len, int32_t S,
                       double* value, void* stream);

/* One job of a batched solve. */
typedef struct {
  xct_plan_t plan;   /* the job's geometry */
  const float* y;    /* device [S][M][N_d] */
  float* x;          /* device [S][n][n]: out (in as well with XCT_CGLS_X0) */
  int32_t S;         /* slices of the job (0: skipped) */
  int32_t reserved;
  double* resid;     /* NULL or device [iters+1][S][2] (as xct_cgls) */
} xct_job;

#define XCT_BATCH_AUTOTUNE 8u  /* time the slice-tile widths per (plan, slices)
                                  and keep the fastest (cached in the plan) */

/*
 * xct_cgls_batch -- `iters` CGLS iterations for every job (each slice its own
 * least-squares problem, Eq. 1 with R = 0), jobs of uneven geometry and slice
 * count solved together: jobs sharing a plan (geometry) are concatenated into
 * one batch of slices (Sec. II-B: slices share A; Sec. III-A2: batches fused
 * into minibatches); every product phase of all geometries with the same
 * kernel configuration is one persistent launch over their combined work; the
 * whole batch runs as one CUDA graph (unless XCT_CGLS_NO_GRAPH).  Flags:
 * XCT_CGLS_X0, XCT_CGLS_NO_GRAPH, XCT_BATCH_AUTOTUNE.  Each job's result is
 * bit-identical to xct_cgls on the concatenation of the slices of all jobs of
 * its plan (same slice-tile width).  A slice whose A^T r_0 is zero stays at
 * its start (no XCT_ERR_BREAKDOWN per job).  Plans must be distinct handles
 * per geometry; a plan appearing in several jobs is one group.  Errors:
 * XCT_ERR_INVALID (bad job, host buffer), XCT_ERR_OOM, XCT_ERR_CUDA,
 * XCT_ERR_TIMEOUT (a bounded wait ran out; results invalid).  Synchronous.
 */
xct_status xct_cgls_batch(const xct_job* jobs, int32_t n_jobs, int32_t iters, uint32_t flags,
                          void* stream);

typedef struct {
  int64_t n_rays, n_pix, nnz;        /* rows of A, columns of A, entries */
  int32_t storage;                   /* xct_dtype */
  int32_t rows_per_block;            /* rows of one thread block */
  int32_t stage_capacity;            /* pixels of A per staged buffer */
  int32_t stage_capacity_at;         /* rays of A^T per staged buffer */
  int64_t stages_a, stages_at;       /* staged buffers over all blocks */
  int64_t slots_a, slots_at;         /* stored entries incl. padding */
  int64_t bytes_a, bytes_at;         /* device bytes of each packed form */
  double plan_ms;                    /* wall time of xct_plan */
  /* filled by the last xct_cgls run with XCT_CGLS_TIMING: */
  double t_project_ms, t_backproject_ms, t_other_ms;
  int64_t n_project, n_backproject;
  /* the parts of t_other_ms: 16-bit staging of the product inputs, vector
     updates (and layout conversions), FP64 scalar kernels */
  double t_stage_ms, t_vector_ms, t_scalar_ms;
  /* 8-byte slots of the paired layouts of A and A^T (XCT_PLAN_PAIRED_ROWS;
     0 without them), padding included */
  int64_t slots_a_paired, slots_at_paired;
  /* staged-row reads of one 64-slice tile on the paired layouts, padding
     aside: the distinct columns of each pair of rows, summed over the stages
     (the plain layouts read one staged row per entry, nnz) */
  int64_t gathers_a_paired, gathers_at_paired;
} xct_stats;

xct_status xct_plan_stats(xct_plan_t plan, xct_stats* out);

/* What xct_plan_export returns. */
#define XCT_EXPORT_A_F64 0      /* A as traced (FP64), needs XCT_PLAN_KEEP_F64 */
#define XCT_EXPORT_AT_F64 1     /* A^T as transposed (FP64), same */
#define XCT_EXPORT_A_STORED 2   /* A decoded from the packed kernel layout:
                                   the stored value, de-normalised */
#define XCT_EXPORT_AT_STORED 3  /* A^T decoded likewise */
#define XCT_EXPORT_A_PAIRED 4   /* A decoded from its paired layout, needs
                                   XCT_PLAN_PAIRED_ROWS (XCT_ERR_INVALID
                                   otherwise, or when the paired layout did
                                   not fit the product kernel's buffers) */
#define XCT_EXPORT_AT_PAIRED 5  /* A^T decoded likewise */

/*
 * xct_plan_export -- copy a matrix to host memory in canonical form: natural
 * row order, natural column ids ascending inside each row.  rowptr: int64
 * [rows+1], col: int32 [nnz], val: double [nnz] (all host).  With rowptr ==
 * NULL only *nnz is written.  Synchronous.  For verification and tooling.
 */
xct_status xct_plan_export(xct_plan_t plan, int32_t what, int64_t* rowptr,
                           int32_t* col, double* val, int64_t* nnz);

/* The pseudo-Hilbert orderings (Sec. III-A1) used by the plan: pix[natural
 * pixel id] = ordered id (n*n entries), ray[natural ray id] = ordered id
 * (M*N_d entries); host int32 arrays, either may be NULL.  Synchronous. */
xct_status xct_plan_order(xct_plan_t plan, int32_t* pix, int32_t* ray);

/*
 * Device memory.  By default the library allocates with cudaMallocAsync /
 * cudaFreeAsync on the call's stream.  A caller may route every allocation
 * through its own allocator (e.g. a framework's caching allocator); the
 * callbacks must be thread-safe and remain valid until reset.  alloc returns
 * NULL on failure (the library then returns XCT_ERR_OOM and frees what it
 * took).  Passing NULL, NULL restores the default.
 */
typedef void* (*xct_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*xct_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
xct_status xct_set_allocator(xct_alloc_fn alloc, xct_free_fn release, void* ctx);

/*
 * xct_project_noalloc -- the projection of xct_project (same arithmetic, same
 * result, bit for bit) for callers that must not allocate device memory
 * during the call: processes whose device memory is owned up front by another
 * component (a serving runtime or a framework allocator that reserved the
 * whole budget) and latency-critical loops where an allocation could block or
 * fail at an unpredictable moment.  The paper has no counterpart; it is a
 * service of this library.
 *
 * All working memory comes from one fixed device array of 32 MiB
 * (33,554,432 bytes).  It becomes resident on a device when xct_plan builds
 * a plan there (its address is looked up then, with the plan's device
 * current), or at the latest on the first xct_project_noalloc call on that
 * device, and stays until the process exits.  With st the slice tile the
 * library picks for S (the least power of two >= S within 8..64 for
 * XCT_F16 / XCT_BF16, 4..32 for XCT_F32, 8..32 for XCT_F16A / XCT_BF16A)
 * and S_pad = st *
 * ceil(S / st), a call needs, each term rounded up to a multiple of 256
 * bytes: 4 * S_pad * n*n (input) + 4 * S_pad * M*N_d (output) + 2 * S_pad *
 * n*n (XCT_F16 and XCT_BF16 only: the 16-bit copy) + 4 * S_pad (per-slice
 * maxima) + 256 (work counter).  A call needing more returns XCT_ERR_INVALID
 * before any work.  x and y must be device pointers (XCT_ERR_INVALID
 * otherwise); the work runs on the plan's device (made current for the call,
 * then restored).  Calls share the array: calls whose GPU work overlaps (on
 * several streams or host threads) race and must be serialised by the
 * caller.  It calls no allocator of any kind.
 */
xct_status xct_project_noalloc(xct_plan_t plan, const float* x, float* y, int32_t S,
                               void* stream);

/*
 * xct_roof_probe -- measures the core roofs of the product kernels on the
 * current GPU (Sec. III-B's register and input reuse bound the product by
 * the FMA and shared-memory rates once the matrix stream is not the limit).
 * Launches ctas_per_sm (1..4) CTAs of 512 threads per SM on `stream`; every
 * thread runs `iters` steps of 4 repetitions of the product's inner step.
 * kind 0: a 16-byte shared-memory gather (8 lanes reading one 128-byte row at
 * a pseudo-random index) feeding 8 mixed-precision FMAs (fma.rn.f32.f16);
 * 1: the 8 mixed FMAs alone; 2: 8 FP32 FMAs alone; 3: the gathers alone;
 * 4: the gather feeding 4 FP32 slices through packed FP32 FMAs.  *ops
 * (host) receives the operation count of the launch: FMAs (kinds 0-2, 4) or
 * 16-byte loads (kind 3); the caller times the launch (CUDA events on
 * `stream`).  Asynchronous.  XCT_ERR_INVALID for kind outside 0..4, iters
 * outside [1, 2^40], ctas_per_sm outside 1..4 or ops == NULL.  The paper has
 * no counterpart (a measurement of this GPU).
 */
xct_status xct_roof_probe(int32_t kind, int64_t iters, int32_t ctas_per_sm, double* ops,
                          void* stream);

/* Thread-local message of the last failing call on this thread. */
const char* xct_last_error(void);

/* Number of kernels this library has launched in the process so far. */
int64_t xct_launch_count(void);

/*
 * xct_set_wait_limit -- wall-time limit of every wait inside the persistent
 * product kernels (a warp waiting for a stage's copies, the producer waiting
 * for a buffer to be released, the block-end rendezvous).  Default 2 s.  A
 * wait that runs out sets the plan's error flag; the kernel lets the copies
 * it already issued land (with its own 2 s limit) and returns, so the GPU
 * context stays usable.  0 makes every wait that is not already satisfied
 * give up at once (a way to exercise this path).  previous: NULL or the
 * limit before the call.  XCT_ERR_INVALID above 60 s.  Process-wide; read
 * at each launch.  The paper has no counterpart.
 */
xct_status xct_set_wait_limit(uint64_t ns, uint64_t* previous);

/*
 * xct_plan_check -- synchronise `stream` and report whether a wait inside a
 * product kernel of this plan ran out since the last check (XCT_ERR_TIMEOUT;
 * the flag is cleared).  Calls that return results to the host, and
 * xct_cgls, xct_cgls_batch and xct_tv_reconstruct, check the flag
 * themselves; products into device buffers are asynchronous and are checked
 * here.
 */
xct_status xct_plan_check(xct_plan_t plan, void* stream);

/* Library version string. */
const char* xct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XCT_H */

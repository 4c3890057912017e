/*
 * C ABI of the GB300 folded-stencil library.
 *
 * The library iterates a constant-coefficient star or box stencil over T time
 * steps on a periodic 1D, 2D or 3D grid (Li et al., "Reducing Redundancy in
 * Data Organization and Arithmetic Calculation for Stencil Computations",
 * Section 1: each point at t+1 is the weighted sum of itself and its
 * neighbours at t), optionally with temporal computation folding (Section 3):
 * m consecutive steps collapse into one sweep of a folded stencil whose
 * weights are the m-fold convolution power of the base weights (Section 3.2
 * folding matrix, Section 3.3 Eq. vfold and Eq. horifold), and with temporal
 * blocking of several folded sweeps per memory round trip (Section 3.4,
 * tessellate tiling and time-loop fusion).
 *
 * Conventions used by every call:
 *  - Orientation: out[p] = sum_o c[o] * in[(p + o) mod shape].
 *  - Grids are dense C-order arrays, shape[0] slowest.
 *  - Coefficients are a dense (2r+1)^ndim array of doubles, axis order
 *    (z, y, x), each axis indexed by offset + r; a star stencil stores zeros
 *    off the axes.
 *  - Every call returns a status; none aborts, exits or traps.  Device-side
 *    waits are bounded; a wait that runs out records STENCIL_ERR_TIMEOUT in
 *    the plan's device status word, which stencil_sync reports.
 *  - A "stream" is a cudaStream_t; NULL means the legacy default stream.
 *  - Calls are not thread-safe on the same plan; one plan is used by one
 *    stream at a time.  Different plans are independent.
 */
#ifndef STENCIL_GB300_H
#define STENCIL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_plan_s *stencil_plan_t;   /* opaque, library-owned */
typedef struct CUstream_st *stencil_stream_t;    /* same type as cudaStream_t */

typedef enum {
    STENCIL_F32 = 0,   /* float  */
    STENCIL_F64 = 1    /* double */
} stencil_dtype_t;

typedef enum {
    STENCIL_OK = 0,
    STENCIL_ERR_INVALID_ARG = 1,   /* bad rank, radius, shape, pointer, T or m      */
    STENCIL_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement   */
    STENCIL_ERR_OOM = 3,           /* a device or host allocation failed            */
    STENCIL_ERR_CUDA = 4,          /* a CUDA runtime or driver call failed          */
    STENCIL_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out            */
    STENCIL_ERR_DEVICE_CHECK = 6   /* a device-side consistency check failed        */
} stencil_status_t;

/* Values of the "precision" option. */
typedef enum {
    STENCIL_PREC_FP32 = 0,    /* CUDA-core FP32 sweeps (default)                          */
    STENCIL_PREC_BF16X3 = 1,  /* folded 2D/3D sweeps on tcgen05: BF16 hi/lo split, 3
                                 products, FP32 accumulation in tensor memory              */
    STENCIL_PREC_BF16X1 = 2,  /* as BF16X3 with the hi*hi product only (error study)      */
    STENCIL_PREC_TF32X3 = 3   /* as BF16X3 with TF32 hi/lo operands (kind::tf32): about 22
                                 significant bits per operand pair instead of 16; folded
                                 radius m*r <= 4                                           */
} stencil_precision_t;

/*
 * Creates a plan for one grid and one base stencil (Section 1).
 *   out_plan  receives the plan; the caller destroys it with stencil_plan_destroy.
 *   ndim      1, 2 or 3.
 *   shape     ndim extents, C order (shape[0] slowest); each >= 2*radius+1.
 *   radius    r >= 1; r <= 4 (CUDA-core sweeps take folded radius m*r <= 16).
 *   coeffs    (2r+1)^ndim doubles as described above; copied, not retained.
 *   dtype     STENCIL_F32 or STENCIL_F64.  FP64 2D/3D grids run FP64 CUDA-core
 *             sweeps (plain or folded, folded radius m*r <= 8 in 2D, <= 4 in
 *             3D; the precision and tensor-core options do not apply to them).
 * The plan binds the CUDA device current at the call.  It computes the FP64
 * folded weights on that device on demand (Section 3.2) and owns all scratch
 * memory, which it allocates on first use.
 * Errors: INVALID_ARG for a bad argument, OOM / CUDA on allocation or device
 * failures.
 */
stencil_status_t stencil_plan(stencil_plan_t *out_plan, int ndim, const int64_t *shape,
                              int radius, const double *coeffs, stencil_dtype_t dtype);

/* Flags of stencil_plan_ex. */
typedef enum {
    STENCIL_FLAG_NONPERIODIC = 1u   /* a non-periodic boundary: not supported, since
                                       folding is exact only on periodic grids      */
} stencil_flags_t;

/*
 * stencil_plan for grids whose rows (and planes) are not densely packed,
 * e.g. a sub-array of a larger allocation or rows padded for alignment (the
 * same problem, Section 1; the layout is the caller's).
 *   pitch_elems  NULL = dense; else ndim-1 strides in elements, C order:
 *                2D {row stride}, 3D {plane stride, row stride}, with
 *                row stride >= shape[ndim-1] and plane stride >= row stride *
 *                shape[1].  Ignored for 1D.  Every in/out grid later given to
 *                stencil_run / stencil_run_batched with this plan uses these
 *                strides; the points between rows and planes are never read
 *                or written.  Host grids use them too.
 *   flags        0 (periodic, the only boundary this library implements) or
 *                STENCIL_FLAG_NONPERIODIC, which returns UNSUPPORTED.
 * Other arguments, ownership and errors as for stencil_plan; additionally
 * INVALID_ARG for pitches below the dense strides or unknown flag bits.
 */
stencil_status_t stencil_plan_ex(stencil_plan_t *out_plan, int ndim, const int64_t *shape,
                                 int radius, const double *coeffs, stencil_dtype_t dtype,
                                 const int64_t *pitch_elems, unsigned flags);

/*
 * Sets a tuning option (all optional).  Keys:
 *   "precision"     stencil_precision_t; the BF16 and TF32 modes run folded 2D and
 *                   3D sweeps (explicit m > 1, m*r <= 8, TF32 m*r <= 4) on the tensor
 *                   cores; plain steps stay on CUDA cores.  A 3D folded sweep is the
 *                   sum over the 2m*r+1 plane offsets dz of the 2D folded sweep with
 *                   that plane slice of c^(m) applied to the plane dz away (Section
 *                   3.3, a 3D grid as a stack of 2D slices): one tensor-core launch
 *                   per offset over all planes, accumulated in the output grid.
 *   "block_b"       temporal-blocking depth: folded sweeps per memory round trip
 *                   (0 = automatic; 1..64, and 2D/3D passes take as many as their
 *                   halo allows).
 *   "tile_y"        rows per CTA tile of the 2D CUDA-core sweep (0 = automatic: 64,
 *                   160 in counterpart form, lowered until the tile fits in shared
 *                   memory).
 *   "stages"        TMA stages per CTA of the 2D CUDA-core sweep, 1..6 (0 =
 *                   automatic: 2, or 1 for blocked passes when two do not fit the
 *                   tile; 1 in counterpart form).  A blocked
 *                   pass refills a stage after the tile's first sweep, and a
 *                   counterpart-form pass after its first vertical fold, so 1
 *                   still overlaps copies with compute; a direct single-sweep
 *                   pass with 1 stage does not.  3D single sweeps: 2 or 3
 *                   stages of four planes (other values: 2).
 *   "cta_threads"   threads per CTA of the 2D CUDA-core sweep: 0 = automatic
 *                   (chosen by the autotuner, else the kernel's own size), 256 =
 *                   two half-size CTAs per SM for folded sweeps that run 512,
 *                   and, on plans[0] of stencil_run_batched, for the batch.
 *   "z_chunk"       3D sweeps: output planes per CTA (or persistent piece), 2..1024
 *                   (0 = automatic: 16 for a single radius-1 sweep, else 32, halved
 *                   down to 8 while the grid has fewer than 4 CTAs per SM).
 *   "tile_1d"       1D sweeps: points per CTA tile, a multiple of 256 in 256..16384
 *                   (0 = automatic: the autotuner's size for fold_m = 0, else 1024
 *                   for overlapped tiles up to folded radius 6 and 4096 above,
 *                   4096 for tessellated FP32 and 1024 for tessellated FP64).
 *   "persistent"    3D CUDA-core runs: 1 = every run of two or more consecutive
 *                   single sweeps of one stencil in ONE persistent launch, whose
 *                   pieces (a 64 x 16 column, one z chunk) start as soon as the
 *                   pieces they read have finished the previous pass, so the
 *                   next pass fills the SMs while a pass drains; 0 = one launch
 *                   per pass; -1 (default) = persistent when a pass has more
 *                   than one and at most 3.5 waves of pieces (grids of about
 *                   192^3 to 320^3, where each pass's last wave leaves SMs
 *                   idle).  Same results either way.  Like the batch queue,
 *                   the persistent launch needs all its CTAs resident at once;
 *                   if other work holds SMs past the wait limit, the run ends
 *                   with TIMEOUT (reported by stencil_sync).
 *   "tc_center"     1 = subtract the grid mean before the BF16 split (default 1).
 *   "center"        2D/3D CUDA-core runs and batches: 1 = store the grid minus its mean
 *                   mu (from an FP64 sum of the input) and add mu * (sum c)^T to the
 *                   output, so that FP32 sums round values near zero rather than near
 *                   mu (default 1; the run is linear, so the result is the same T
 *                   steps); 0 = store the values as they are.
 *   "counterparts"  2D CUDA-core sweeps in counterpart form (Section 3.3 vertical then
 *                   horizontal folding; Section 3.5 counterpart reuse): when c^(m)
 *                   factors exactly as a sum of K <= 2 separable terms u_k (x) v_k, a
 *                   sweep folds the input vertically with each u_k and combines the
 *                   results horizontally with the v_k, 2K(2R+1) multiply-adds per
 *                   point.  0 = when that undercuts the nonzeros of c^(m) and the
 *                   sweep is folded (m >= 2) or wide (R >= 3) (default); 1 = always
 *                   (UNSUPPORTED when the rank is above 2);
 *                   2 = never.  Folded radii 1, 2, 3, 4, 6, 8.
 *   "tc_form"       tensor-core kernel: 1 = one MMA per row offset of the folded
 *                   weights (the row shift applied through the operand descriptor);
 *                   2 = four row offsets per MMA, the remaining shifts done in the
 *                   epilogue (fewer, wider MMAs; 125-row tiles); 0 = by the folded
 *                   radius: grouped from R = m*r >= 6 (default).
 *   "tc_tma_store"  1 = per-offset tensor-core tiles leave through a TMA store when the
 *                   destination allows it (default 1); 0 = direct stores.
 *   "tessellate"    1D passes: 1 = exact tessellate tiling (Section 3.4): per pass of b
 *                   steps, tiles first advance their shrinking triangles, then the
 *                   inverted triangles around the tile boundaries finish every point,
 *                   with no step computed twice (two launches per pass; used where
 *                   the tile of 2048 FP64 / 4096 FP32 points is at least 2*b*R wide);
 *                   0 = overlapped tiles that recompute their rim (default).  The
 *                   autotuner tries both.
 *   "wait_limit_ms" bound of every device-side wait (default 2000).
 *   "autotune"      1 = time candidates when stencil_run gets fold_m = 0 (default 1).
 *   "graph"         1 = capture each distinct run (pointers, T, m, options) once into
 *                   a CUDA graph and replay it (default 1); 0 = launch kernel by kernel.
 *                   A run on a stream that is itself being captured is never graphed.
 *   "fault_withhold_copy"  test hook: 1 = the 2D CUDA-core sweep and both 3D kernels
 *                   never issue a CTA's first copy, so their bounded waits run out
 *                   and stencil_sync reports STENCIL_ERR_TIMEOUT (no GPU fault; the
 *                   context stays usable).
 *   "fault_withhold_dep"   test hook: 1 = in a batched run led by this plan, or in
 *                   this plan's persistent 3D launch, every dependency on a
 *                   previous pass counts as unmet, so the bounded dependency
 *                   wait runs out (TIMEOUT, as above).
 *   "fault_withhold_mma"   test hook: 1 = the tensor-core kernels' MMA issuer stops
 *                   before its first MMA, so the other roles' bounded waits run out
 *                   (TIMEOUT, as above; tensor memory is still freed).
 * Errors: INVALID_ARG for an unknown key or an out-of-range value.
 */
stencil_status_t stencil_plan_set_option(stencil_plan_t plan, const char *key, int64_t value);

/*
 * Reads a plan property.  Keys: "last_m", "last_b", "last_engine" (0 CUDA core,
 * 1 tensor core), "last_tile_y" (rows per tile of the last 2D CUDA-core run's
 * first pass, or points per tile of the last 1D run), "last_tc_form" (1 per-offset, 2 grouped: the tensor-core kernel
 * of the last tensor-core run), "last_cp" (separable terms K of the last 2D
 * CUDA-core run's folded passes in counterpart form, 0 = direct form),
 * "last_tess" (1 if the last 1D run's first pass was tessellated exactly),
 * "last_threads" (threads per CTA of the last stencil_run_batched launch: 512,
 * or 256 for two CTAs per SM; or of the first pass of the last 2D CUDA-core
 * run), "last_stages" (TMA stages per CTA of that pass), "last_persistent"
 * (1 if the last 3D CUDA-core
 * run took its single sweeps in one persistent multi-pass launch),
 * "launches" (kernels the plan has launched so far),
 * "scratch_bytes" (device bytes the plan owns).
 */
stencil_status_t stencil_plan_get(stencil_plan_t plan, const char *key, int64_t *value);

/*
 * Advances `in` by T steps into `out` (Section 1 time loop; Section 3 folding).
 *   in, out   prod(shape) elements of the plan's dtype.  Either both device
 *             pointers or both host pointers (pageable or pinned).  With host
 *             pointers the call copies in and out through plan-owned device
 *             buffers and returns after the result is in `out`.  in == out is
 *             allowed.  `in` is only read.  The caller keeps ownership.
 *   T         time steps, >= 0 (T = 0 copies).
 *   fold_m    1 = plain sweeps; m > 1 = floor(T/m) folded sweeps of the m-fold
 *             convolution power plus T mod m plain steps; 0 = let the
 *             autotuner choose m (and the blocking depth), cached per
 *             (ndim, shape, radius, coefficients, dtype, GPU).
 *   stream    the stream all work is ordered on.  With device pointers the
 *             call is asynchronous.
 * Errors: INVALID_ARG (null pointers, T < 0, fold_m < 0, folded radius wider
 * than the grid), UNSUPPORTED (folding a stencil or precision this build has
 * no kernel for), CUDA on a failed launch.
 */
stencil_status_t stencil_run(stencil_plan_t plan, const void *in, void *out, int64_t T,
                             int fold_m, stencil_stream_t stream);

/*
 * Advances n independent grids in one persistent launch fed by a device work
 * queue (a CUDA graph is captured once per set of plans and replayed).
 *   plans     n plans, each 2D FP32 of radius 1 or 2, created on the current
 *             device.
 *   in, out   n device pointers each (grids in the matching plan's layout,
 *             pitched where the plan was made by stencil_plan_ex).
 *   T         n step counts (>= 0).
 *   fold_m    n fold factors (1 plain, > 1 folded, 0 automatic) or NULL for 0.
 *             A fold the batched kernel lacks is lowered to the largest it
 *             has (the result is the same T steps).  With 0 and no block_b
 *             option on the grid's plan, the fold and blocking depth come from
 *             the batch autotuner, which times each class of grids (radius,
 *             pattern, floor(log2 area)) and caches its choices per batch
 *             composition (the set of classes) and GPU, so that one batch's
 *             choice for a class never seeds another batch; it also picks the
 *             batch's tile height unless plans[0] sets
 *             the "tile_y" option, which then pins it (at most 128 rows), and
 *             the CTA shape: 512 threads, one CTA per SM, or 256 threads, two
 *             per SM with tiles that fit half an SM's shared memory (pinned
 *             by "cta_threads" 256 on plans[0]).
 * Grids must not alias one another.  Errors as for stencil_run; a timed-out
 * dependency wait is reported by stencil_sync on plans[0] (the launch needs
 * all its CTAs resident at once: other work holding SMs past the wait limit
 * ends it that way).
 */
stencil_status_t stencil_run_batched(int n, const stencil_plan_t *plans,
                                     const void *const *in, void *const *out,
                                     const int64_t *T, const int *fold_m,
                                     stencil_stream_t stream);

/*
 * Waits for `stream` and returns the plan's device status (TIMEOUT or
 * DEVICE_CHECK if a kernel recorded one since the last sync), then clears it.
 */
stencil_status_t stencil_sync(stencil_plan_t plan, stencil_stream_t stream);

/*
 * Copies the FP64 folded weights c^(m) (Section 3.2) the plan computed on the
 * GPU into host_out, which holds n >= (2*m*r+1)^ndim doubles (dense, centred).
 * Synchronous.  Errors: INVALID_ARG for m < 1 or n too small.
 */
stencil_status_t stencil_folded_coeffs(stencil_plan_t plan, int m, double *host_out, size_t n);

/*
 * Relative L2 error on the GPU, accumulated in FP64:
 *   host_out[0] = ||y - ref|| / ||ref||,
 *   host_out[1] = the same after removing each array's mean.
 *   y         n device elements of type ydtype; ref: n device doubles.
 * Synchronises `stream`.  Uses temporary device memory from the stream-ordered
 * allocator.  Errors: INVALID_ARG for null pointers or n < 1.
 */
stencil_status_t stencil_rel_l2(const void *y, stencil_dtype_t ydtype, const double *ref,
                                int64_t n, double *host_out, stencil_stream_t stream);

/*
 * Host-only planner counts of the scalar profitability analysis (Section 3.2,
 * Eq. ce, Eq. uce, Eq. pi) for folding m steps of the given stencil:
 *   out[0] = |C(E)|  : instructions of the naive m-step expression, i.e.
 *            |S| * sum_{s<m} |support(c^(s))| (each intermediate point is a
 *            |S|-way weighted sum);
 *   out[1] = |C(E_lambda)| : taps of the folded stencil, |support(c^(m))|.
 * The profitable index is out[0] / out[1].  Needs no GPU.
 */
stencil_status_t stencil_fold_cost(int ndim, int radius, const double *coeffs, int m,
                                   int64_t *out);

/*
 * Host-only counterpart factorisation (Section 3.3, Eq. vfold and Eq. horifold;
 * Section 3.5) of W x W folded 2D weights `folded` (row-major, row offset
 * slowest): the smallest K with folded[a][b] = sum_{k<K} u_k[a] v_k[b], found
 * by Gaussian elimination with complete pivoting in FP64 (entries below 1e-12
 * of the largest count as zero).  Writes K to *k_out and K rows of W values to
 * u_out (the counterparts' vertical weights) and v_out (their horizontal
 * weights); both must hold max_k * W doubles.  When the rank exceeds max_k,
 * *k_out = max_k + 1 and the first max_k terms are written.  Needs no GPU.
 * Errors: INVALID_ARG for W outside 1..17, max_k outside 1..W, or a
 * null pointer.
 */
stencil_status_t stencil_fold_counterparts(int W, const double *folded, int max_k, int *k_out,
                                           double *u_out, double *v_out);

/*
 * Host-only schedule of the exact tessellate tiling (Section 3.4) that the
 * "tessellate" option runs: for one tile of W points in a line of such tiles,
 * b steps of a radius-R stencil, stage1[i] and stage2[i] receive how many of
 * the b steps point i takes in the triangle stage and in the inverted-triangle
 * stage (they sum to b).  W = 9, b = 4, R = 1 gives 0,1,2,3,4,3,2,1,0 and
 * 4,3,2,1,0,1,2,3,4.  stage1 and stage2 hold W ints each.  Needs no GPU.
 * Errors: INVALID_ARG for W < 2*b*R, b < 1, R < 1 or a null pointer.
 */
stencil_status_t stencil_tessellation_counts(int W, int b, int R, int *stage1, int *stage2);

/*
 * T plain steps of a 1D periodic stencil without allocating any memory.
 * The paper has no counterpart of this call: it serves callers that cannot
 * call cudaMalloc -- code inside a framework whose own allocator owns all
 * device memory, and deployments that must not touch the allocator after
 * start-up.  stencil_run needs a plan, which allocates; this call does not.
 *   in, out   n device elements of `dtype` (F32 or F64); in == out allowed.
 *   n         points, 2*radius+1 <= n and n * sizeof(dtype) <= 16 MiB.
 *   radius    1, 2, 3, 4, 6, 8, 12 or 16.
 *   coeffs    2*radius+1 host doubles (offsets -radius..radius); copied.
 *   T         steps, >= 0.
 * The intermediate grid lives in one fixed 16 MiB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  All calls share the array and each call fully
 * overwrites what it reads back, so nothing needs clearing, but calls whose
 * work overlaps on the GPU (other streams, other threads) race on it.
 * Asynchronous on `stream`.  Allocates nothing: no cudaMalloc, no cudaFree.
 * Errors: INVALID_ARG for bad arguments or a grid above 16 MiB,
 * UNSUPPORTED for another radius, CUDA on a failed launch.
 */
stencil_status_t stencil_run_1d_noalloc(const void *in, void *out, int64_t n, int radius,
                                        const double *coeffs, int64_t T, stencil_dtype_t dtype,
                                        stencil_stream_t stream);

/* Frees the plan and everything it owns.  Waits for the plan's work first. */
void stencil_plan_destroy(stencil_plan_t plan);

/* Static name of a status code. */
const char *stencil_status_string(stencil_status_t status);

/* Detail of the last error on the calling thread ("" if none). */
const char *stencil_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_GB300_H */

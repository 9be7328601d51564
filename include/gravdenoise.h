/*
 * gravdenoise.h -- C ABI of the GB300 (sm_103a) adaptive dual-weight
 * gravitational point-cloud denoiser (arXiv 2512.10386, Sec. 3).
 *
 * The problem statement (Sec. 3): given a cloud P = {p_1 .. p_N} of xyz
 * points, partition it with an octree into leaves {P_t} (Eq. 10), remove
 * isolated points with an adaptive voxel occupancy gate in each leaf
 * (Eq. 11-12), remove low-density points with a kNN density percentile gate
 * (Eq. 13-14), score the survivors with the density/distance dual-weight
 * gravitational sum (Eq. 15-21), keep the best of each leaf and return the
 * union of the leaves' survivors (Eq. 22).  Here the result is a per-point
 * keep mask in input order, plus the scores and the stage that removed each
 * point.
 *
 * Conventions shared by every call:
 *  - Points are float32 xyz, array-of-structures [n][3] (12 bytes a point).
 *  - Buffers may be host or device pointers; the library detects which
 *    (cudaPointerGetAttributes).  Host buffers are staged through the
 *    context's device memory, in stream order on the given stream: pinned
 *    (page-locked, mapped) host input is read in place by the first kernel,
 *    which writes the device copy; other host input is copied first.  Host
 *    outputs are filled at the end of the call: pinned ones by a kernel that
 *    stores through their mapped addresses (any byte offset), others by the
 *    copy engine.  Pinned host memory keeps all of it asynchronous.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *    of a call is ordered on that stream.
 *  - The caller owns every buffer it passes; the context owns all scratch.
 *  - Calls on one context are not thread-safe: use one context per host
 *    thread, or serialise.  Different contexts are independent.
 *  - Return value: DENOISE_OK (0) or a negative DENOISE_E_* status.
 */
#ifndef GRAVDENOISE_H
#define GRAVDENOISE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DENOISE_OK 0
#define DENOISE_E_INVAL (-1)     /* bad argument or parameter                          */
#define DENOISE_E_NONFINITE (-2) /* a coordinate is NaN or Inf (rejected, not filtered) */
#define DENOISE_E_CAPACITY (-3)  /* more points or frames than the context was made for */
#define DENOISE_E_NOMEM (-4)     /* device or pinned allocation failed                  */
#define DENOISE_E_TIMEOUT (-5)   /* a bounded device-side wait ran out                  */
#define DENOISE_E_CUDA (-6)      /* a CUDA runtime call failed                          */
#define DENOISE_E_STATE (-7)     /* call out of order (e.g. backward without forward)   */

/* Selection rule of the last step. */
#define DENOISE_SELECT_TOPRATIO 0u  /* keep the best ceil(lambda*|P_2|) of each leaf (Sec. 3, end) */
#define DENOISE_SELECT_THRESHOLD 1u /* keep ln F_i >= tau (differentiable form)                   */

/*
 * Method parameters.  Every field is read on every call.  Values the paper
 * states are noted; the others are unstated there and are readings.  The
 * "without octree" configuration of Table 8 is leaf_capacity >= n (one leaf).
 */
typedef struct denoise_params {
  uint32_t k;              /* K neighbours, 1..64 (paper default 12; Eq. 13, Sec. 4.3.1)        */
  uint32_t leaf_capacity;  /* max points per octree leaf, >= 1 (Sec. 3)                         */
  uint32_t max_depth;      /* octree depth limit 0..21, the minimum leaf side rule (Sec. 3)     */
  float beta;              /* voxel enlargement coefficient > 0 (Eq. 11)                        */
  uint32_t min_vox_count;  /* n_v, minimum voxel occupancy (Eq. 12; paper 4)                    */
  float rho_percentile;    /* q in percent, 0..100, MATLAB prctile units (Eq. 14; paper 0.2)    */
  float alpha;             /* density weighting index (Eq. 17)                                  */
  float sigma;             /* distance-weight scale > 0, sigma_i = sigma * r_K,i (Eq. 18-19)    */
  float gamma;             /* kernel exponent > 0: 1/((d^2)^(gamma/2) + eps_k); paper 2 (Eq. 20)*/
  float eps_rho;           /* epsilon of Eq. 17, >= 0                                           */
  float eps_k;             /* epsilon of Eq. 20, >= 0                                           */
  uint32_t select_mode;    /* DENOISE_SELECT_TOPRATIO or DENOISE_SELECT_THRESHOLD               */
  float lambda;            /* Top-lambda keep ratio in (0, 1] (Sec. 3, end)                     */
  float tau;               /* log-score threshold of the THRESHOLD rule                         */
  float temperature;       /* soft-mask temperature T > 0 (differentiable form only)            */
  uint32_t stage_off;      /* structural ablations of Sec. 4.3.2 (Table 9), 0 = the method:    */
                           /*  bit 0 no voxel gate (A1): every point of a leaf is in P_1;      */
                           /*  bit 1 no density gate (A2): P_2 = P_1, and a lone point of a    */
                           /*        leaf is scored (F = 0) instead of removed;                */
                           /*  bit 2 no score selection (A3): every point of P_2 is kept with  */
                           /*        score 0 (with bit 1 also set, no kNN is computed)         */
  uint32_t rescore_p2;     /* 1: the score uses a kNN recomputed within P_2 (its own k_eff,    */
                           /*    r_K, densities and rho_med): the other reading of Eq. 21;     */
                           /*    0 = the kNN on P_1 (Sec. 3's single N x K table)              */
  uint32_t cross_leaf;     /* 1: kNN candidates are the P_1 points of the 27 octree cells of   */
                           /*    the leaf's level around the leaf's cell, not the leaf alone;  */
                           /*    the gates, median and selection stay per leaf.  Needs        */
                           /*    denoise_set_cross_leaf(ctx, 1); not combined with stage_off  */
                           /*    or rescore_p2.  0 = within the leaf (Sec. 3)                  */
} denoise_params;

typedef struct denoise_ctx denoise_ctx;

/*
 * Create a context on CUDA device `device` able to process up to
 * `max_points` points in one call, split into at most `max_frames` frames.
 * All device scratch of the forward path (sort buffers, octree leaf table,
 * per-leaf spill space) is allocated here, sized for max_points; the forward
 * calls (denoise_run, denoise_run_batch, denoise_run_debug) allocate no device
 * memory.  Two optional features allocate later, on request: the training
 * cache, made by the first denoise_set_training(ctx, 1) (about 520 bytes a
 * point), and the cross-leaf kNN tables, made by the first
 * denoise_set_cross_leaf(ctx, 1) (about 265 bytes a point); the metric and
 * baseline calls use the context's scratch and allocate nothing.  The largest buffer
 * is allocated first, so a context too large for the GPU fails with E_NOMEM
 * before it holds any memory.  *out receives the context (NULL on failure).
 * Errors: E_INVAL (out NULL, max_points or max_frames 0), E_NOMEM, E_CUDA.
 */
int denoise_create(denoise_ctx **out, int device, size_t max_points, uint32_t max_frames);

/* Release a context and all its memory.  NULL is a no-op.  Waits for the
 * context's outstanding work first. */
int denoise_destroy(denoise_ctx *ctx);

/* Static English text for a status code. */
const char *denoise_strerror(int status);

/*
 * Denoise one cloud (Sec. 3, Eq. 10-22).
 *  xyz   [n][3] float32, host or device.
 *  mask  [n] uint8, 1 = keep (the point belongs to P_denoise, Eq. 22); may be NULL.
 *  score [n] float32, F_i (Eq. 21) for points of P_2, 0 otherwise; may be NULL.
 *  stage [n] uint8: 0 kept, 1 removed by the voxel gate (Eq. 12), 2 removed
 *        by the density gate (Eq. 14, or a leaf too small for a neighbour),
 *        3 removed by the score selection; may be NULL.
 * n = 0 is a valid no-op.  In synchronous mode (the default, see
 * denoise_set_sync) the call returns after the results are in place and
 * reports device-side errors (E_NONFINITE, E_TIMEOUT); in asynchronous mode
 * it returns once the work is enqueued and denoise_get_status reports them.
 * Errors: E_INVAL, E_NONFINITE, E_CAPACITY, E_TIMEOUT, E_CUDA.
 */
int denoise_run(denoise_ctx *ctx, const float *xyz, size_t n, const denoise_params *p,
                uint8_t *mask, float *score, uint8_t *stage, void *stream);

/*
 * Denoise `nframes` independent clouds in one pass.  The clouds are
 * concatenated in `xyz` ([offsets[nframes]][3]); frame f owns points
 * offsets[f] .. offsets[f+1]-1.  `offsets` is a HOST array of nframes+1
 * non-decreasing values starting at 0.  mask/score/stage follow the same
 * concatenated layout.  Each frame is denoised exactly as denoise_run would
 * denoise it alone.  With graphs enabled (denoise_set_graphs) the whole batch
 * runs as one captured CUDA graph, re-captured only when the frame layout,
 * the buffers or the parameters change.
 * Errors: as denoise_run; E_CAPACITY if nframes > max_frames.
 */
int denoise_run_batch(denoise_ctx *ctx, const float *xyz, const uint64_t *offsets, uint32_t nframes,
                      const denoise_params *p, uint8_t *mask, float *score, uint8_t *stage,
                      void *stream);

/* Execution options of a context. */
int denoise_set_sync(denoise_ctx *ctx, int synchronous);   /* default 1                     */
int denoise_set_graphs(denoise_ctx *ctx, int enable);      /* default 0 (direct launches)   */
int denoise_set_profiling(denoise_ctx *ctx, int enable);   /* per-stage CUDA events, default 0 */

/*
 * Execution tuning (results do not depend on it).
 *  leaf_ctas_per_sm  how many persistent CTAs of the fused per-leaf kernel run
 *                    per SM; 0 (default) = as many as fit.
 *  leaf_smem_points  largest leaf (in points) that the per-leaf kernel keeps in
 *                    shared memory; larger leaves take its global-memory path.
 *                    A smaller value shrinks each CTA's shared memory so that
 *                    more CTAs fit per SM.  Rounded down to a power of two,
 *                    at least 64; 0 (default) = the leaf capacity.
 *  leaf_threads      threads of a per-leaf CTA: 64 or 128 (0 = default 128).
 *                    64 suits workloads of many small leaves (fewer idle
 *                    warps per leaf); other values give E_INVAL.
 * The autotuner (paper_2512_10386_gb300/autotune.py) picks both together with
 * the leaf capacity, which is a method parameter.
 * Errors: E_INVAL for a NULL context or tuning pointer, or leaf_threads not 0, 64 or 128.
 */
typedef struct denoise_tuning {
  uint32_t leaf_ctas_per_sm;
  uint32_t leaf_smem_points;
  uint32_t leaf_threads;
} denoise_tuning;
int denoise_set_tuning(denoise_ctx *ctx, const denoise_tuning *t);

/*
 * Evaluation metrics of Sec. 4.1 between a clean (ground-truth) cloud A and a
 * denoised cloud B, both float32 xyz [n][3], host or device:
 *  metrics[0] = MSE of Eq. 29: the mean over A of the squared distance from
 *               each clean point to its nearest point of B (the paper takes the
 *               nearest neighbour as the corresponding point);
 *  metrics[1] = Chamfer distance of Eq. 30: that mean plus the mean over B of the
 *               squared distance to the nearest point of A;
 *  metrics[2] = PSNR of Eq. 29, 10 log10(M^2 / MSE), M = the diagonal of A's
 *               bounding box (the paper's usual choice for M).
 * `metrics` is a HOST double[3].  nn_clean [n_clean] / nn_denoised
 * [n_denoised] (host or device, may be NULL) receive the per-point nearest
 * squared distances.  Every pair of points is compared (exact nearest
 * neighbours); squared distances are FP32 with the method's operation order,
 * the means FP64 in a fixed order (deterministic).
 * Errors: E_INVAL (NULL argument, an empty cloud), E_CAPACITY (a cloud larger
 * than max_points), E_NONFINITE, E_TIMEOUT, E_CUDA.
 */
int denoise_eval_metrics(denoise_ctx *ctx, const float *clean, size_t n_clean, const float *denoised,
                         size_t n_denoised, double *metrics, float *nn_clean, float *nn_denoised, void *stream);

/*
 * The gravitational-function baseline of Sec. 2.2 (Eq. 1-9), the paper's
 * comparison method: centroid theta (Eq. 1), extents H (Eq. 2), radius
 * R = 6 (HxHy + HxHz + HyHz) / N (Eq. 3), d_i = |p_i - theta| (Eq. 4),
 * n_i = number of points within R of p_i, itself included (Eq. 5),
 * F_i = G n_i / d_i^2 (Eq. 6), T = alpha G (Hx + Hy + Hz) / N (Eq. 7); a point is
 * kept iff F_i >= T / d_i (Eq. 8-9).  The paper sets G = 6.67e-11 and
 * alpha = 600.  Eq. 3 is not scale-free (an area over a count), so the result
 * depends on the units of the coordinates, as in the paper.
 *  xyz [n][3] float32, host or device; mask [n] uint8 (1 = keep), host or
 *  device; n_i [n] uint32 counts (may be NULL); params HOST double[5] =
 *  (theta_x, theta_y, theta_z, R, T) (may be NULL).
 * The neighbour test compares the FP32 squared distance (the method's
 * operation order) with R^2; every pair is compared.
 * Errors: E_INVAL (NULL argument, n = 0, G or alpha not positive and finite),
 * E_CAPACITY (n > max_points), E_NONFINITE, E_TIMEOUT, E_CUDA.
 */
int denoise_run_baseline(denoise_ctx *ctx, const float *xyz, size_t n, double G, double alpha, uint8_t *mask,
                         uint32_t *n_i, double *params, void *stream);

/*
 * Bounded device-side waits.  Two waits in the path can spin: a radix-sort
 * tile waiting for its predecessor's published prefix (decoupled look-back)
 * and the leaf kernel waiting for its bulk copy of a leaf.  Each gives up after
 * `iterations` polls (0 = the built-in limit, 2^22), sets the call's status to
 * DENOISE_E_TIMEOUT and returns, so the call ends and the context stays usable.
 * Errors: E_INVAL for a NULL context.
 */
int denoise_set_wait_limit(denoise_ctx *ctx, uint32_t iterations);

/*
 * Test hook for the timeout path (no paper counterpart; off by default).  With
 * tile >= 0, tile `tile` of the first radix-sort pass of every later call on
 * this context never publishes its look-back prefix, so the tile after it waits
 * until the wait limit (denoise_set_wait_limit) runs out and the call returns
 * DENOISE_E_TIMEOUT with void results.  No memory is touched out of bounds and
 * nothing waits without a limit.  tile = -1 turns the hook off.
 * Errors: E_INVAL for a NULL context or tile < -1.
 */
int denoise_test_hold_lookback(denoise_ctx *ctx, int32_t tile);

/* Wait for the context's last call on `stream` and return its device-side
 * status (DENOISE_OK, E_NONFINITE or E_TIMEOUT). */
int denoise_get_status(denoise_ctx *ctx, void *stream);

/* Statistics of the last completed call (valid after it finished). */
typedef struct denoise_stats {
  uint64_t n_points;     /* points processed                                          */
  uint64_t n_leaves;     /* octree leaves                                             */
  uint64_t knn_pairs;    /* sum over leaves of |P_1|(|P_1|-1): candidate pairs scanned */
  uint64_t n_p1;         /* points that passed the voxel gate                         */
  uint64_t n_p2;         /* points that passed the density gate                       */
  uint64_t score_terms;  /* neighbour terms summed by the score, sum over P_2 of k_eff  */
  uint32_t launches;     /* kernels launched by the call                              */
  uint32_t n_stages;     /* entries valid in stage_ms                                 */
  float stage_ms[8];     /* with profiling: init+bbox+keys, sort, leaf finder, leaf prep, fused leaf kernel */
} denoise_stats;

int denoise_get_stats(denoise_ctx *ctx, denoise_stats *out);

/*
 * Per-stage intermediates for parity checks.  Every pointer may be NULL;
 * all are DEVICE pointers, per point in input order unless noted.
 */
typedef struct denoise_debug {
  uint64_t *key;         /* [n] 63-bit Morton key of the point (root cube of its frame)   */
  uint32_t *leaf_start;  /* [n] sorted position (within the frame) of its leaf's first point */
  uint32_t *leaf_count;  /* [n] N_t of its leaf                                            */
  float *leaf_h;         /* [n] adaptive voxel size h of its leaf (Eq. 11)                 */
  uint32_t *vox_count;   /* [n] occupancy of its voxel (Eq. 12)                            */
  float *r2;             /* [n] floored squared distance to the k-th neighbour, P_1 only   */
  uint32_t *nbr;         /* [n][k] neighbour indices (input order), 0xFFFFFFFF padding     */
  float *nbr_d2;         /* [n][k] squared neighbour distances (FP32), 0 padding           */
  double *leaf_rho_med;  /* [n] rho_med of its leaf (Eq. 16), 0 if the leaf scores nobody  */
} denoise_debug;

/* denoise_run with intermediates written to `dbg` (may be NULL). */
int denoise_run_debug(denoise_ctx *ctx, const float *xyz, size_t n, const denoise_params *p,
                      uint8_t *mask, float *score, uint8_t *stage, const denoise_debug *dbg,
                      void *stream);

/*
 * Differentiable form (reading of Sec. 3 for calibration; the paper itself
 * only thresholds).  With training enabled, the forward keeps, for every
 * scored point, its neighbour list and density terms on the device.
 *  denoise_soft_removal: removal probability r_i = 1 - sigmoid((ln F_i - tau)/T)
 *    for points of P_2 and 1 for points removed by the gates, for the last
 *    forward call and its parameters; removal [n] float32 (host or device).
 *  denoise_backward: given dL/dr_i ([n] float32, host or device) for the last
 *    forward call, accumulate dL/d(alpha, sigma, gamma, tau) into grad4
 *    (HOST double[4], overwritten), with the neighbour sets, gates and
 *    densities held fixed (none of them depends on these four parameters).
 *    Reductions are in FP64 with a fixed order: results are deterministic.
 * Errors: E_STATE if the last forward did not run with training enabled.
 */
int denoise_set_training(denoise_ctx *ctx, int enable);  /* default 0 */

/*
 * Cross-leaf kNN (denoise_params.cross_leaf).  The first denoise_set_cross_leaf
 * (ctx, 1) allocates the variant's per-point tables (neighbour positions for
 * K = 64, r_K^2, k_eff and a P_1 flag: about 265 bytes a point for max_points);
 * later forward calls allocate nothing.  A call with cross_leaf = 1 on a context
 * without them fails with E_STATE.
 * Errors: E_INVAL (NULL context), E_NOMEM, E_CUDA.
 */
int denoise_set_cross_leaf(denoise_ctx *ctx, int enable);
int denoise_soft_removal(denoise_ctx *ctx, float *removal, void *stream);
int denoise_backward(denoise_ctx *ctx, const float *grad_removal, double *grad4, void *stream);

/*
 * No-allocation variant of denoise_run.  The paper has no counterpart: this
 * call exists for callers that cannot allocate device memory at all -- for
 * example code that runs under a host framework which owns every device
 * allocation, or inside a real-time loop whose policy forbids cudaMalloc.
 * It denoises one cloud of at most DENOISE_NOALLOC_MAX_POINTS points with
 * exactly the kernels of denoise_run, but all scratch lives in one
 * file-scope device array of the library (6,570,752 bytes per GPU, held by every
 * GPU that loads the library until the process exits).  Nothing is allocated:
 * no context, no cudaMalloc/cudaFree, no pinned memory.
 *  xyz   [n][3] float32, DEVICE pointer of the current GPU (host pointers and
 *        pointers of another GPU are rejected).
 *  mask, score, stage: as denoise_run, DEVICE pointers or NULL.
 *  Works on the calling thread's current CUDA device.  The first call on a
 *  device looks up the scratch array's device address (cudaGetSymbolAddress).
 *  Each call synchronises `stream` and returns the device-side status, so no
 *  call can be recorded into a CUDA graph: a call on a stream that is being
 *  captured returns E_INVAL and enqueues nothing.
 *  All calls share the one scratch array, and it keeps the last call's
 *  contents (the call clears what must start at zero): calls that overlap on
 *  the GPU -- from two host threads, or on two streams -- race and must not
 *  be made.
 * Errors: E_INVAL (NULL, host or other-GPU xyz/outputs, bad parameters, a
 * capturing stream), E_CAPACITY (n > DENOISE_NOALLOC_MAX_POINTS), E_NONFINITE,
 * E_TIMEOUT, E_CUDA.
 */
#define DENOISE_NOALLOC_MAX_POINTS 16384u
int denoise_run_noalloc(const float *xyz, size_t n, const denoise_params *p, uint8_t *mask, float *score,
                        uint8_t *stage, void *stream);
/* Size in bytes of denoise_run_noalloc's scratch array (6,570,752); 0 if the
 * library was built inconsistently (the array would not cover the kernels'
 * needs, and denoise_run_noalloc then fails with E_INVAL).  Host-only: needs
 * no GPU. */
size_t denoise_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* GRAVDENOISE_H */

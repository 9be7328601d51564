/*
 * oracle.h -- plain FP64 CPU reference of the adaptive dual-weight
 * gravitational point-cloud denoiser (arXiv 2512.10386, Sec. 3, Eq. 10-22).
 *
 * TEST INFRASTRUCTURE ONLY.  This file and oracle.c are the checker that the
 * GPU library is compared against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may call it; the product path never
 * links or calls it.  It shares no code, header, table or helper with the
 * CUDA library: every definition here is written independently.
 */
#ifndef GRAV_ORACLE_H
#define GRAV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Method parameters (names follow the paper's notation). */
typedef struct {
  uint32_t k;              /* K, neighbours per point (Sec. 3, Eq. 13)              */
  uint32_t leaf_capacity;  /* max points per octree leaf (Sec. 3)                   */
  uint32_t max_depth;      /* octree depth limit <= 21 (min leaf side, Sec. 3)      */
  float beta;              /* voxel enlargement coefficient (Eq. 11)                */
  uint32_t min_vox_count;  /* n_v, minimum voxel occupancy (Eq. 12)                 */
  float rho_percentile;    /* q, in percent as MATLAB prctile (Eq. 14)              */
  float alpha;             /* density weighting index (Eq. 17)                      */
  float sigma;             /* global distance-weight scale (Eq. 18)                 */
  float gamma;             /* gravitational kernel exponent, 2 in the paper (Eq. 20)*/
  float eps_rho;           /* epsilon of Eq. 17                                     */
  float eps_k;             /* epsilon of Eq. 20                                     */
  uint32_t select_mode;    /* 0: per-leaf Top-lambda (Sec. 3 end), 1: ln F >= tau   */
  float lambda;            /* Top-lambda keep ratio                                 */
  float tau;               /* log-score threshold (mode 1)                          */
  float temperature;       /* soft-mask temperature (differentiable form)           */
  uint32_t stage_off;      /* ablations (Table 9): bit 0 no voxel gate (A1), bit 1 no density
                              gate (A2), bit 2 no score selection (A3); 0 = the method         */
  uint32_t rescore_p2;     /* 1: the score uses a kNN recomputed within P_2               */
  uint32_t cross_leaf;     /* 1: kNN candidates from the 27 same-level cells around the leaf */
} orc_params;

/* Outputs; every pointer may be NULL.  Per-point arrays are in input order. */
typedef struct {
  uint8_t *mask;        /* [n] 1 = keep                                          */
  uint8_t *stage;       /* [n] 0 kept, 1 voxel gate, 2 density gate, 3 score    */
  double *score;        /* [n] F_i for points of P_2, else 0                     */
  uint64_t *key;        /* [n] 63-bit Morton key                                 */
  uint32_t *leaf_of;    /* [n] leaf index (leaves numbered in Morton order)      */
  uint32_t *vox_count;  /* [n] occupancy of the point's voxel (Eq. 12)           */
  float *r2;            /* [n] floored squared k-th neighbour distance, P_1 only */
  double *rho;          /* [n] kNN density (Eq. 13), P_1 only                    */
  uint32_t *nbr;        /* [n][k] neighbour input indices, 0xFFFFFFFF padding    */
  float *nbr_d2;        /* [n][k] squared distances (FP32), 0 padding            */
  int64_t *n_leaves;    /* number of leaves                                      */
  uint32_t *leaf_start; /* [n] first sorted position of each leaf                */
  uint32_t *leaf_count; /* [n] N_t                                               */
  uint32_t *leaf_level; /* [n] octree level of each leaf                         */
  float *leaf_lo;       /* [n][3] leaf bounding-box minimum (voxel grid origin)  */
  float *leaf_h;        /* [n] adaptive voxel size h (Eq. 11)                    */
  double *leaf_rho_med; /* [n] rho_med over P_2 of the leaf (Eq. 16)             */
  uint32_t *leaf_n1;    /* [n] |P_1| of the leaf                                 */
  uint32_t *leaf_n2;    /* [n] |P_2| of the leaf                                 */
  float *root;          /* [4] root cube: lo_x, lo_y, lo_z, side                 */
} orc_out;

/* Status codes. */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENONFINITE -2
#define ORC_ENOMEM -3

/* Full pipeline (octree -> voxel gate -> kNN + density gate -> score -> select). */
int orc_denoise(const float *xyz, int64_t n, const orc_params *p, orc_out *out);
/* The same, with the (independent) leaves spread over `threads` host threads
 * when the library is built with OpenMP: for timing the oracle on all cores. */
int orc_denoise_threads(const float *xyz, int64_t n, const orc_params *p, orc_out *out, int threads);

/* Soft-F1 loss of the differentiable form and its gradient with respect to
 * (alpha, sigma, gamma, tau).  noise[i] = 1 marks a noise point; in_loss (may
 * be NULL = all points) selects the points that enter the loss sums.
 * removal (may be NULL) receives the soft removal probability of each point. */
int orc_softf1(const float *xyz, int64_t n, const orc_params *p, const uint8_t *noise,
               const uint8_t *in_loss, double *loss, double grad[4], double *removal);

/* Evaluation metrics (Sec. 4.1, Eq. 29-30), FP64, brute force.
 * orc_nn_d2: out[i] = min over j of ||a_i - b_j||^2.
 * orc_metrics: with A = the clean cloud and B = the denoised cloud,
 *   mse = mean over A of the squared distance to the nearest point of B
 *         (the "corresponding point" of Eq. 29 is that nearest neighbour),
 *   cd  = Eq. 30: mse + mean over B of the squared distance to the nearest point of A,
 *   psnr = 10 log10(M^2 / mse), M = diagonal of A's bounding box.
 * Both sets must be non-empty (ORC_EINVAL otherwise). */
int orc_nn_d2(const float *a, int64_t na, const float *b, int64_t nb, double *out);
int orc_metrics(const float *clean, int64_t na, const float *den, int64_t nb, double *mse, double *cd,
                double *psnr);

/* The gravitational-function baseline of Sec. 2.2 (Eq. 1-9).
 *   centroid theta (Eq. 1), extents H (Eq. 2), radius R = 6(HxHy + HxHz + HyHz)/N (Eq. 3),
 *   d_i = ||p_i - theta|| (Eq. 4), n_i = |{p_j : ||p_j - p_i|| <= R}| with p_i itself
 *   counted (Eq. 5), F_i = G n_i / d_i^2 (Eq. 6), T = alpha G (Hx + Hy + Hz) / N (Eq. 7),
 *   keep iff F_i >= T / d_i (Eq. 8-9).
 * The neighbour test compares the FP32 squared distance (the method's fixed
 * operation order) with R^2 in FP64.  Every output pointer may be NULL except keep. */
int orc_baseline(const float *xyz, int64_t n, double G, double alpha, uint8_t *keep, uint32_t *n_i,
                 double *d_i, double *F_i, double *R_out, double *T_out);

/* Cube root used for Eq. 11: fixed Newton sequence in FP64 (see oracle.c). */
double orc_cbrt_spec(double u);

/* Morton key of one quantised triple (bit 3b+2 <- x, 3b+1 <- y, 3b <- z). */
uint64_t orc_interleave(uint32_t qx, uint32_t qy, uint32_t qz);

#ifdef __cplusplus
}
#endif
#endif

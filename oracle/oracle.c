/*
 * oracle.c -- plain, slow FP64 CPU reference of the adaptive dual-weight
 * gravitational denoiser of arXiv 2512.10386 (Sec. 3, Eq. 10-22).
 *
 * TEST INFRASTRUCTURE ONLY: the checker the GPU library is compared against.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may call it.  It shares no code with the CUDA library.
 *
 * Arithmetic: FP64 everywhere, except where a step is *defined* on FP32 values
 * so that its integer outcome (Morton key, voxel index, neighbour order,
 * density-gate rank) is reproducible bit for bit on any IEEE machine.  Those
 * steps spell out every FP32 operation; the file must be compiled with
 * -ffp-contract=off and without fast-math so no operation is fused or
 * reordered.  Algorithms are the obvious ones: qsort for every ordering,
 * brute force for every count and every neighbour search.
 *
 * Readings of the paper where it is silent, garbled or ambiguous (each one
 * also listed in the design notes):
 *  R1 root cube: axis-aligned bounding cube anchored at the FP32 minimum,
 *     side = largest FP32 extent (1 if all points coincide); coordinates are
 *     quantised to 21 bits per axis, q = min(2^21-1, floor((x-lo)*s)),
 *     s = 2^21/side, all in FP32.
 *  R2 octree: node (level L, top 3L key bits) is a leaf iff it holds at most
 *     leaf_capacity points or L = max_depth (the minimum-side rule); empty
 *     children are skipped; leaves are numbered in Morton order.
 *  R3 leaf extents are floored at delta = side*2^-21 per axis so that flat or
 *     colinear leaves keep V_t > 0 (Eq. 10).
 *  R4 Eq. 11's cube root is the fixed Newton sequence of orc_cbrt_spec.
 *  R5 voxel grid origin = leaf bounding-box minimum; voxel index per axis
 *     floor((x-lo_t)/h) in FP32, saturated at 2^21-1; Eq. 12 uses ">= n_v".
 *  R6 kNN searches the leaf's P_1 only, excludes the point itself, uses
 *     k_eff = min(K, |P_1|-1) (a leaf with |P_1| <= 1 loses its points at the
 *     density gate), d^2 = fma(dz,dz,fma(dy,dy,dx*dx)) in FP32 with
 *     dx = x_j - x_i, and orders candidates by (d^2, input index).
 *  R7 r_K^2 is the k_eff-th squared distance floored at delta^2 (FP32);
 *     Eq. 13 uses k_eff for K.
 *  R8 Eq. 14: q is in percent (MATLAB prctile units); prctile is taken per
 *     leaf over P_1 and evaluated exactly: keep rho_i >= rho_(c) with
 *     c = clamp(ceil(n*q/100 + 0.5), 1, n) on ascending rho, which is what
 *     the hazen-interpolated percentile gives in exact arithmetic.
 *  R9 Eq. 16: rho_med is the median over the leaf's P_2 (mean of the two
 *     middle values for an even count).
 *  R10 Eq. 21 reuses the single kNN pass on P_1: N_K(i), r_K and rho_j come
 *     from it, so a neighbour j may lie outside P_2.  Eq. 20 is generalised
 *     to 1/((d^2)^(gamma/2) + eps_k); gamma = 2 is the paper's kernel.
 *     Scores are summed in FP64 in neighbour order.
 *  R11 Top-lambda (end of Sec. 3): keep ceil(lambda*|P_2|) points of each
 *     leaf by (F descending, input index ascending).  Mode 1 instead keeps
 *     ln F >= tau (the differentiable form).
 *  R13 structural variants (ablations of Sec. 4.3.2): see process_leaf.
 *  R12 differentiable form: removal probability r_i = 1 - sigmoid((ln F_i -
 *     tau)/T) on P_2 and 1 elsewhere; soft-F1 = 2 sum(r y)/(sum r + sum y)
 *     (Eq. 26-28 with soft counts); loss = 1 - soft-F1.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 2097151u                    /* 2^21 - 1                      */
#define INV_TWO21 4.76837158203125e-07f  /* 2^-21, exact in FP32          */
#define NONE32 0xFFFFFFFFu
#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* orderings (qsort comparators)                                       */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t idx; } keyed_t;

static int cmp_keyed(const void *a, const void *b) {
  const keyed_t *x = (const keyed_t *)a, *y = (const keyed_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

typedef struct { float d2; uint32_t idx; uint32_t pos; } cand_t;

static int cmp_cand(const void *a, const void *b) {
  const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
  if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x < y) ? -1 : (x > y) ? 1 : 0;
}

typedef struct { double f; uint32_t idx; uint32_t pos; } ranked_t;

static int cmp_ranked(const void *a, const void *b) {  /* F desc, index asc */
  const ranked_t *x = (const ranked_t *)a, *y = (const ranked_t *)b;
  if (x->f != y->f) return x->f > y->f ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* R1: Morton keys                                                     */
/* ------------------------------------------------------------------ */
uint64_t orc_interleave(uint32_t qx, uint32_t qy, uint32_t qz) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
    key |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
    key |= (uint64_t)((qz >> b) & 1u) << (3 * b);
  }
  return key;
}

static uint32_t quantise(float x, float lo, float s) {
  float d = x - lo;
  float t = d * s;
  float f = floorf(t);
  return (f < 2097151.0f) ? (uint32_t)f : QMAX;
}

/* ------------------------------------------------------------------ */
/* R4: cube root for Eq. 11.  u = m * 2^e with m in [0.5, 1) (frexp);  */
/* start at y = 2^floor(e/3) and take 10 Newton steps on y^3 - u = 0,   */
/* y <- y - (y*y*y - u) / (3*(y*y)), each operation rounded in FP64.    */
/* ------------------------------------------------------------------ */
double orc_cbrt_spec(double u) {
  int e = 0;
  (void)frexp(u, &e);
  int k = (e >= 0) ? e / 3 : -((-e + 2) / 3);
  double y = ldexp(1.0, k);
  for (int it = 0; it < 10; ++it) {
    double y2 = y * y;
    double y3 = y2 * y;
    double num = y3 - u;
    double den = 3.0 * y2;
    y = y - num / den;
  }
  return y;
}

/* ------------------------------------------------------------------ */
/* R2: octree leaves over the sorted keys (recursive, top-down)        */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t start, count, level; } leaf_t;

typedef struct {
  const keyed_t *sorted;
  uint32_t cap, max_depth;
  leaf_t *leaves;
  int64_t n_leaves;
} octree_t;

static void octree_build(octree_t *o, uint32_t level, uint32_t begin, uint32_t end) {
  uint32_t count = end - begin;
  if (count <= o->cap || level == o->max_depth) {
    leaf_t lf = {begin, count, level};
    o->leaves[o->n_leaves++] = lf;
    return;
  }
  int shift = 3 * (21 - (int)(level + 1));  /* child triple of level+1 */
  uint32_t i = begin;
  for (uint32_t c = 0; c < 8; ++c) {
    uint32_t j = i;
    while (j < end && (uint32_t)((o->sorted[j].key >> shift) & 7u) == c) ++j;
    if (j > i) octree_build(o, level + 1, i, j);
    i = j;
  }
}

/* ------------------------------------------------------------------ */
/* per-leaf pipeline                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
  const float *xyz;
  const orc_params *p;
  float delta;         /* side * 2^-21 */
  orc_out *out;
  double *dF;          /* [n][3] dF/d(alpha, sigma, gamma), or NULL */
  double *F_all;       /* [n] scores (internal, always filled)     */
  uint8_t *stage_all;  /* [n] stages (internal, always filled)     */
} ctx_t;

static float coord(const ctx_t *c, uint32_t i, int a) { return c->xyz[3 * (size_t)i + a]; }

static float sq_dist(const ctx_t *c, uint32_t i, uint32_t j) {
  float dx = coord(c, j, 0) - coord(c, i, 0);
  float dy = coord(c, j, 1) - coord(c, i, 1);
  float dz = coord(c, j, 2) - coord(c, i, 2);
  float xx = dx * dx;
  return fmaf(dz, dz, fmaf(dy, dy, xx));
}

/* R6, R7 and Eq. 13 for every point of a list: its k_eff nearest among the
 * others of the list (positions into the list), the floored k_eff-th squared
 * distance and the density.  With `record`, the debug outputs are written. */
static int knn_list(ctx_t *c, const uint32_t *pts, uint32_t n1, uint32_t keff, uint32_t *nb, float *nd2,
                    float *r2, double *rho, int record) {
  const orc_params *p = c->p;
  orc_out *o = c->out;
  cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * n1);
  if (!cand) return ORC_ENOMEM;
  const uint32_t *p1 = pts;
  const float delta2 = c->delta * c->delta;
  for (uint32_t a = 0; a < n1; ++a) {
    uint32_t m = 0;
    for (uint32_t b = 0; b < n1; ++b) {
      if (b == a) continue;
      cand[m].d2 = sq_dist(c, p1[a], p1[b]);
      cand[m].idx = p1[b];
      cand[m].pos = b;
      ++m;
    }
    qsort(cand, m, sizeof(cand_t), cmp_cand);
    for (uint32_t s = 0; s < keff; ++s) {
      nb[(size_t)a * keff + s] = cand[s].pos;
      nd2[(size_t)a * keff + s] = cand[s].d2;
    }
    float rk2 = cand[keff - 1].d2;
    r2[a] = (rk2 < delta2) ? delta2 : rk2;
    /* Eq. 13 */
    double rr = (double)r2[a];
    rho[a] = (double)keff / ((4.0 / 3.0) * PI_D * (rr * sqrt(rr)));
    if (!record) continue;
    if (o->r2) o->r2[p1[a]] = r2[a];
    if (o->rho) o->rho[p1[a]] = rho[a];
    if (o->nbr)
      for (uint32_t s = 0; s < p->k; ++s)
        o->nbr[(size_t)p1[a] * p->k + s] = (s < keff) ? cand[s].idx : NONE32;
    if (o->nbr_d2)
      for (uint32_t s = 0; s < p->k; ++s)
        o->nbr_d2[(size_t)p1[a] * p->k + s] = (s < keff) ? cand[s].d2 : 0.0f;
  }
  free(cand);
  return ORC_OK;
}

/* Structural variants (Sec. 4.3.2, Tables 8-9), reading R13:
 *  stage_off bit 0: no voxel gate (A1): P_1 = the leaf's points;
 *  stage_off bit 1: no density gate (A2): P_2 = P_1, and a point with no
 *                   possible neighbour is scored (F = 0) instead of removed;
 *  stage_off bit 2: no score selection (A3): every point of P_2 is kept, with
 *                   score 0; without A2 as well, no kNN is computed at all;
 *  rescore_p2:      the score uses a second kNN computed within P_2 (its own
 *                   k_eff, r_K and densities, and rho_med over them) instead of
 *                   the kNN on P_1 (the other reading of Eq. 21).
 * "Without octree" (Table 8) is leaf_capacity >= N: the root is the only leaf. */
/* Eq. 10-12 for one leaf: extents, voxel size h, voxel occupancy and the voxel
 * gate.  p1 [count] receives P_1 (input indices, leaf order); returns |P_1|, or
 * -1 when out of memory. */
static int64_t voxel_gate(ctx_t *c, const keyed_t *sorted, const leaf_t *lf, uint32_t leaf_id, uint32_t *p1) {
  const orc_params *p = c->p;
  orc_out *o = c->out;
  const int a1_on = !(p->stage_off & 1u);
  const uint32_t nt = lf->count;
  uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * nt);
  uint32_t *vox = (uint32_t *)malloc(sizeof(uint32_t) * nt * 3);
  uint32_t *cnt = (uint32_t *)malloc(sizeof(uint32_t) * nt);
  if (!idx || !vox || !cnt) return -1;
  for (uint32_t t = 0; t < nt; ++t) idx[t] = sorted[lf->start + t].idx;

  /* Eq. 10 with R3: leaf bounding box, extents floored at delta */
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) { lo[a] = coord(c, idx[0], a); hi[a] = lo[a]; }
  for (uint32_t t = 1; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      float v = coord(c, idx[t], a);
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
  float H[3];
  for (int a = 0; a < 3; ++a) {
    H[a] = hi[a] - lo[a];
    if (H[a] < c->delta) H[a] = c->delta;
  }
  double V = (double)H[0] * (double)H[1] * (double)H[2];
  /* Eq. 11 with R4 */
  double u = V / (double)nt;
  float h = (float)((double)p->beta * orc_cbrt_spec(u));

  /* Eq. 12 with R5: voxel indices, occupancy by brute-force comparison */
  for (uint32_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      float d = coord(c, idx[t], a) - lo[a];
      float q = d / h;
      float f = floorf(q);
      vox[3 * t + a] = (f < 2097151.0f) ? (uint32_t)f : QMAX;
    }
  uint32_t n1 = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    if (o->leaf_of) o->leaf_of[idx[t]] = leaf_id;
    if (!a1_on) {  /* the voxel gate is off: every point is in P_1 */
      if (o->vox_count) o->vox_count[idx[t]] = 0;
      p1[n1++] = idx[t];
      continue;
    }
    uint32_t k = 0;
    for (uint32_t s = 0; s < nt; ++s)
      k += (vox[3 * s] == vox[3 * t] && vox[3 * s + 1] == vox[3 * t + 1] &&
            vox[3 * s + 2] == vox[3 * t + 2]);
    cnt[t] = k;
    if (o->vox_count) o->vox_count[idx[t]] = k;
    if (k >= p->min_vox_count) p1[n1++] = idx[t];
    else c->stage_all[idx[t]] = 1;
  }
  if (o->leaf_lo) for (int a = 0; a < 3; ++a) o->leaf_lo[3 * (size_t)leaf_id + a] = lo[a];
  if (o->leaf_h) o->leaf_h[leaf_id] = h;
  if (o->leaf_n1) o->leaf_n1[leaf_id] = n1;
  if (o->leaf_n2) o->leaf_n2[leaf_id] = 0;
  if (o->leaf_rho_med) o->leaf_rho_med[leaf_id] = 0.0;

  free(idx); free(vox); free(cnt);
  return n1;
}

static int process_leaf(ctx_t *c, const keyed_t *sorted, const leaf_t *lf, uint32_t leaf_id) {
  const orc_params *p = c->p;
  orc_out *o = c->out;
  const int a2_on = !(p->stage_off & 2u), a3_on = !(p->stage_off & 4u);
  uint32_t *p1 = (uint32_t *)malloc(sizeof(uint32_t) * lf->count);
  if (!p1) return ORC_ENOMEM;
  const int64_t g1 = voxel_gate(c, sorted, lf, leaf_id, p1);
  if (g1 < 0) return ORC_ENOMEM;
  const uint32_t n1 = (uint32_t)g1;
  uint32_t *idx = NULL, *vox = NULL, *cnt = NULL;  /* (kept by voxel_gate) */

  if (!a2_on && !a3_on) {  /* neither gate nor score needs a neighbour: P_1 is kept */
    if (o->leaf_n2) o->leaf_n2[leaf_id] = n1;
    free(idx); free(vox); free(cnt); free(p1);
    return ORC_OK;
  }
  if (n1 <= 1 && a2_on) {  /* R6: not enough support for a neighbour */
    for (uint32_t t = 0; t < n1; ++t) c->stage_all[p1[t]] = 2;
    free(idx); free(vox); free(cnt); free(p1);
    return ORC_OK;
  }

  /* kNN on P_1 (R6, R7) */
  const uint32_t keff = (n1 <= 1) ? 0 : (p->k < n1 - 1) ? p->k : n1 - 1;
  const size_t nk = (size_t)n1 * (keff ? keff : 1);
  uint32_t *nb = (uint32_t *)malloc(sizeof(uint32_t) * nk);   /* P_1 positions */
  float *nd2 = (float *)malloc(sizeof(float) * nk);
  float *r2 = (float *)malloc(sizeof(float) * n1);
  double *rho = (double *)malloc(sizeof(double) * n1);
  double *sorted_rho = (double *)malloc(sizeof(double) * n1);
  uint8_t *in2 = (uint8_t *)malloc(n1);
  if (!nb || !nd2 || !r2 || !rho || !sorted_rho || !in2) return ORC_ENOMEM;
  if (keff && knn_list(c, p1, n1, keff, nb, nd2, r2, rho, 1)) return ORC_ENOMEM;

  /* Eq. 14 with R8: exact hazen percentile of rho over the leaf's P_1 */
  uint32_t m2 = 0;
  if (a2_on) {
    memcpy(sorted_rho, rho, sizeof(double) * n1);
    qsort(sorted_rho, n1, sizeof(double), cmp_double);
    double pos = (double)n1 * (double)p->rho_percentile / 100.0 + 0.5;
    double cc = ceil(pos);
    uint32_t crank = (cc < 1.0) ? 1u : (cc > (double)n1) ? n1 : (uint32_t)cc;
    double thr = sorted_rho[crank - 1];
    for (uint32_t a = 0; a < n1; ++a) {
      in2[a] = rho[a] >= thr;
      if (in2[a]) sorted_rho[m2++] = rho[a];
      else c->stage_all[p1[a]] = 2;
    }
  } else {
    for (uint32_t a = 0; a < n1; ++a) {
      in2[a] = 1;
      if (keff) sorted_rho[m2] = rho[a];
      ++m2;
    }
  }
  if (o->leaf_n2) o->leaf_n2[leaf_id] = m2;
  if (!a3_on) {  /* no score selection: P_2 is kept */
    free(sorted_rho); free(in2);
    free(nb); free(nd2); free(r2); free(rho);
    free(idx); free(vox); free(cnt); free(p1);
    return ORC_OK;
  }

  /* The set the score runs on: P_1 with the P_2 flags (reading R10), or P_2
   * alone with its own kNN (rescore_p2). */
  uint32_t ns = n1, ks = keff;
  uint32_t *set = p1;
  uint32_t *p2 = NULL;
  if (p->rescore_p2) {
    p2 = (uint32_t *)malloc(sizeof(uint32_t) * (m2 ? m2 : 1));
    if (!p2) return ORC_ENOMEM;
    uint32_t t2 = 0;
    for (uint32_t a = 0; a < n1; ++a)
      if (in2[a]) p2[t2++] = p1[a];
    ns = m2;
    ks = (ns <= 1) ? 0 : (p->k < ns - 1) ? p->k : ns - 1;
    if (ks && knn_list(c, p2, ns, ks, nb, nd2, r2, rho, 1)) return ORC_ENOMEM;
    for (uint32_t a = 0; a < ns; ++a) {
      in2[a] = 1;
      sorted_rho[a] = rho[a];
    }
    set = p2;
  }

  /* Eq. 16 with R9: median of rho over P_2 */
  double rho_med = 0.0;
  if (ks) {
    qsort(sorted_rho, m2, sizeof(double), cmp_double);
    rho_med = (m2 & 1u) ? sorted_rho[(m2 - 1) / 2]
                        : 0.5 * (sorted_rho[m2 / 2 - 1] + sorted_rho[m2 / 2]);
  }
  if (o->leaf_rho_med) o->leaf_rho_med[leaf_id] = rho_med;

  /* Eq. 15-21 with R10: dual-weight gravitational score (an empty neighbour set scores 0) */
  const double alpha = p->alpha, sigma = p->sigma, gamma = p->gamma;
  const double eps_rho = p->eps_rho, eps_k = p->eps_k;
  const double wden_den = rho_med * rho_med + eps_rho;
  ranked_t *rk = (ranked_t *)malloc(sizeof(ranked_t) * (m2 ? m2 : 1));
  if (!rk) return ORC_ENOMEM;
  uint32_t r = 0;
  for (uint32_t a = 0; a < ns; ++a) {
    if (!in2[a]) continue;
    double F = 0.0, dA = 0.0, dS = 0.0, dG = 0.0;
    const double r2i = ks ? (double)r2[a] : 0.0;
    for (uint32_t s = 0; s < ks; ++s) {
      uint32_t b = nb[(size_t)a * ks + s];
      double d2 = (double)nd2[(size_t)a * ks + s];
      double W = rho[a] * rho[b] / wden_den;                      /* Eq. 17 base */
      double w_den = pow(W, alpha / 2.0);                         /* Eq. 17      */
      double w_dis = exp(-d2 / (2.0 * (sigma * sigma) * r2i));    /* Eq. 18-19   */
      double D = pow(d2, gamma / 2.0);
      double kern = 1.0 / (D + eps_k);                            /* Eq. 20      */
      double t = w_den * w_dis * kern;                            /* Eq. 15, 21  */
      F += t;
      if (c->dF) {
        dA += t * 0.5 * log(W);
        dS += t * d2 / (sigma * sigma * sigma * r2i);
        if (d2 > 0.0) dG += -t * D * 0.5 * log(d2) / (D + eps_k);
      }
    }
    c->F_all[set[a]] = F;
    if (c->dF) {
      c->dF[3 * (size_t)set[a] + 0] = dA;
      c->dF[3 * (size_t)set[a] + 1] = dS;
      c->dF[3 * (size_t)set[a] + 2] = dG;
    }
    rk[r].f = F;
    rk[r].idx = set[a];
    rk[r].pos = a;
    ++r;
  }

  /* R11: selection */
  if (p->select_mode == 0) {
    qsort(rk, m2, sizeof(ranked_t), cmp_ranked);
    double want = ceil((double)p->lambda * (double)m2);
    uint32_t keep = (want > (double)m2) ? m2 : (uint32_t)want;
    for (uint32_t t = 0; t < m2; ++t) c->stage_all[rk[t].idx] = (t < keep) ? 0 : 3;
  } else {
    for (uint32_t t = 0; t < m2; ++t)
      c->stage_all[rk[t].idx] = (log(rk[t].f) >= (double)p->tau) ? 0 : 3;
  }

  free(rk); free(sorted_rho); free(in2); free(p2);
  free(nb); free(nd2); free(r2); free(rho);
  free(idx); free(vox); free(cnt); free(p1);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* R14: cross-leaf kNN.  The candidates of the points of a leaf at level L */
/* are the P_1 points of the 27 octree cells of level L around (and       */
/* including) the leaf's own cell: neighbours come from adjacent cells    */
/* too, so a point near a leaf's border is not cut off from the points    */
/* across it.  Densities are per point (each from its own kNN); the       */
/* percentile gate, the median and the selection stay per leaf, and the   */
/* score of a point uses its neighbours' own densities with the rho_med   */
/* of the point's leaf.                                                   */
/* ------------------------------------------------------------------ */
static uint32_t deinterleave(uint64_t key, int axis) {  /* axis 0: x (bit 3b+2), 1: y, 2: z */
  uint32_t q = 0;
  for (int b = 0; b < 21; ++b) q |= (uint32_t)((key >> (3 * b + 2 - axis)) & 1u) << b;
  return q;
}

static int64_t lower_key(const keyed_t *sorted, int64_t n, uint64_t key) {  /* first position with key >= key */
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (sorted[mid].key < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

static int run_cross_leaf(ctx_t *c, const keyed_t *sorted, int64_t n, const leaf_t *leaves, int64_t n_leaves) {
  const orc_params *p = c->p;
  orc_out *o = c->out;
  uint8_t *in1 = (uint8_t *)calloc((size_t)n, 1);           /* by input index */
  uint32_t *leaf_of = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *lp1 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *keff_of = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
  uint32_t *nbi = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * p->k); /* neighbour input indices */
  float *nd2 = (float *)malloc(sizeof(float) * (size_t)n * p->k);
  float *r2 = (float *)calloc((size_t)n, sizeof(float));
  double *rho = (double *)calloc((size_t)n, sizeof(double));
  uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  cand_t *cl = (cand_t *)malloc(sizeof(cand_t) * (size_t)n);
  if (!in1 || !leaf_of || !lp1 || !keff_of || !nbi || !nd2 || !r2 || !rho || !cand || !cl) return ORC_ENOMEM;
  /* Eq. 10-12 per leaf: P_1 */
  for (int64_t L = 0; L < n_leaves; ++L) {
    const int64_t g1 = voxel_gate(c, sorted, &leaves[L], (uint32_t)L, lp1);
    if (g1 < 0) return ORC_ENOMEM;
    for (int64_t t = 0; t < g1; ++t) in1[lp1[t]] = 1;
    for (uint32_t t = 0; t < leaves[L].count; ++t) leaf_of[sorted[leaves[L].start + t].idx] = (uint32_t)L;
  }
  const float delta2 = c->delta * c->delta;
  /* the kNN of every P_1 point among the P_1 points of its leaf's 27-cell block */
  for (int64_t L = 0; L < n_leaves; ++L) {
    const leaf_t *lf = &leaves[L];
    const uint32_t lv = lf->level;
    const int sh = 3 * (21 - (int)lv);
    const uint64_t k0 = sorted[lf->start].key;
    const int64_t cx = deinterleave(k0, 0) >> (21 - lv), cy = deinterleave(k0, 1) >> (21 - lv),
                  cz = deinterleave(k0, 2) >> (21 - lv);
    const int64_t side = (int64_t)1 << lv;
    uint32_t nc = 0;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          const int64_t x = cx + dx, y = cy + dy, z = cz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) continue;
          const uint64_t pre = orc_interleave((uint32_t)x, (uint32_t)y, (uint32_t)z);  /* level-lv cell */
          const uint64_t kb = (sh >= 64) ? 0 : pre << sh, ke = (sh >= 64) ? ~0ull : (pre + 1) << sh;
          int64_t a = lower_key(sorted, n, kb);
          const int64_t b = (lv == 0) ? n : lower_key(sorted, n, ke);
          for (; a < b; ++a)
            if (in1[sorted[a].idx]) cand[nc++] = sorted[a].idx;
        }
    for (uint32_t t = 0; t < lf->count; ++t) {
      const uint32_t i = sorted[lf->start + t].idx;
      if (!in1[i] || nc <= 1) continue;
      const uint32_t keff = (p->k < nc - 1) ? p->k : nc - 1;
      uint32_t m = 0;
      for (uint32_t u = 0; u < nc; ++u) {
        if (cand[u] == i) continue;
        cl[m].d2 = sq_dist(c, i, cand[u]);
        cl[m].idx = cand[u];
        cl[m].pos = u;
        ++m;
      }
      qsort(cl, m, sizeof(cand_t), cmp_cand);
      for (uint32_t s2 = 0; s2 < keff; ++s2) {
        nbi[(size_t)i * p->k + s2] = cl[s2].idx;
        nd2[(size_t)i * p->k + s2] = cl[s2].d2;
      }
      keff_of[i] = keff;
      float rk2 = cl[keff - 1].d2;
      r2[i] = (rk2 < delta2) ? delta2 : rk2;
      double rr = (double)r2[i];
      rho[i] = (double)keff / ((4.0 / 3.0) * PI_D * (rr * sqrt(rr)));  /* Eq. 13 */
      if (o->r2) o->r2[i] = r2[i];
      if (o->rho) o->rho[i] = rho[i];
      if (o->nbr)
        for (uint32_t s2 = 0; s2 < p->k; ++s2) o->nbr[(size_t)i * p->k + s2] = (s2 < keff) ? cl[s2].idx : NONE32;
      if (o->nbr_d2)
        for (uint32_t s2 = 0; s2 < p->k; ++s2) o->nbr_d2[(size_t)i * p->k + s2] = (s2 < keff) ? cl[s2].d2 : 0.0f;
    }
  }
  /* per leaf: Eq. 14 gate, Eq. 16 median, Eq. 15-21 score, selection */
  double *srt = (double *)malloc(sizeof(double) * (size_t)n);
  ranked_t *rk = (ranked_t *)malloc(sizeof(ranked_t) * (size_t)n);
  if (!srt || !rk) return ORC_ENOMEM;
  for (int64_t L = 0; L < n_leaves; ++L) {
    const leaf_t *lf = &leaves[L];
    uint32_t n1 = 0;
    for (uint32_t t = 0; t < lf->count; ++t) {
      const uint32_t i = sorted[lf->start + t].idx;
      if (!in1[i]) continue;
      if (!keff_of[i]) { c->stage_all[i] = 2; continue; }  /* no candidate besides itself */
      lp1[n1++] = i;
    }
    if (o->leaf_n2) o->leaf_n2[L] = 0;
    if (o->leaf_rho_med) o->leaf_rho_med[L] = 0.0;
    if (!n1) continue;
    for (uint32_t a = 0; a < n1; ++a) srt[a] = rho[lp1[a]];
    qsort(srt, n1, sizeof(double), cmp_double);
    double pos = (double)n1 * (double)p->rho_percentile / 100.0 + 0.5;
    double cc = ceil(pos);
    uint32_t crank = (cc < 1.0) ? 1u : (cc > (double)n1) ? n1 : (uint32_t)cc;
    double thr = srt[crank - 1];
    uint32_t m2 = 0;
    for (uint32_t a = 0; a < n1; ++a) {
      if (rho[lp1[a]] >= thr) {  /* P_2, compacted in place (m2 <= a) */
        srt[m2] = rho[lp1[a]];
        lp1[m2] = lp1[a];
        ++m2;
      } else {
        c->stage_all[lp1[a]] = 2;
      }
    }
    qsort(srt, m2, sizeof(double), cmp_double);
    double rho_med = (m2 & 1u) ? srt[(m2 - 1) / 2] : 0.5 * (srt[m2 / 2 - 1] + srt[m2 / 2]);
    if (o->leaf_rho_med) o->leaf_rho_med[L] = rho_med;
    if (o->leaf_n2) o->leaf_n2[L] = m2;
    const double alpha = p->alpha, sigma = p->sigma, gamma = p->gamma;
    const double wden_den = rho_med * rho_med + p->eps_rho, eps_k = p->eps_k;
    for (uint32_t a = 0; a < m2; ++a) {
      const uint32_t i = lp1[a];
      double F = 0.0;
      const double r2i = (double)r2[i];
      for (uint32_t s2 = 0; s2 < keff_of[i]; ++s2) {
        const uint32_t j = nbi[(size_t)i * p->k + s2];
        const double d2 = (double)nd2[(size_t)i * p->k + s2];
        const double W = rho[i] * rho[j] / wden_den;                          /* Eq. 17 base */
        const double kern = 1.0 / (pow(d2, gamma / 2.0) + eps_k);             /* Eq. 20      */
        F += pow(W, alpha / 2.0) * exp(-d2 / (2.0 * (sigma * sigma) * r2i)) * kern;  /* Eq. 15-21 */
      }
      c->F_all[i] = F;
      rk[a].f = F;
      rk[a].idx = i;
      rk[a].pos = a;
    }
    if (p->select_mode == 0) {
      qsort(rk, m2, sizeof(ranked_t), cmp_ranked);
      double want = ceil((double)p->lambda * (double)m2);
      uint32_t keep = (want > (double)m2) ? m2 : (uint32_t)want;
      for (uint32_t t = 0; t < m2; ++t) c->stage_all[rk[t].idx] = (t < keep) ? 0 : 3;
    } else {
      for (uint32_t t = 0; t < m2; ++t) c->stage_all[rk[t].idx] = (log(rk[t].f) >= (double)p->tau) ? 0 : 3;
    }
  }
  free(srt); free(rk);
  free(in1); free(leaf_of); free(lp1); free(keff_of); free(nbi); free(nd2); free(r2); free(rho); free(cand); free(cl);
  return ORC_OK;
}

static int check_params(const orc_params *p) {
  if (!p) return ORC_EINVAL;
  if (p->k == 0 || p->k > 64) return ORC_EINVAL;
  if (p->leaf_capacity == 0) return ORC_EINVAL;
  if (p->max_depth > 21) return ORC_EINVAL;
  if (!(p->beta > 0.0f) || !isfinite(p->beta)) return ORC_EINVAL;
  if (!(p->rho_percentile >= 0.0f && p->rho_percentile <= 100.0f)) return ORC_EINVAL;
  if (!(p->lambda > 0.0f && p->lambda <= 1.0f)) return ORC_EINVAL;
  if (!(p->gamma > 0.0f) || !isfinite(p->gamma)) return ORC_EINVAL;
  if (!(p->sigma > 0.0f) || !isfinite(p->sigma)) return ORC_EINVAL;
  if (!isfinite(p->alpha) || !(p->eps_rho >= 0.0f) || !(p->eps_k >= 0.0f)) return ORC_EINVAL;
  if (p->select_mode > 1) return ORC_EINVAL;
  if (!(p->temperature > 0.0f)) return ORC_EINVAL;
  if (p->stage_off > 7u || p->rescore_p2 > 1u || p->cross_leaf > 1u) return ORC_EINVAL;
  if (p->cross_leaf && (p->stage_off || p->rescore_p2)) return ORC_EINVAL;  /* not combined (R14) */
  return ORC_OK;
}

static int run(const float *xyz, int64_t n, const orc_params *p, orc_out *o, double *dF,
               double *F_all, uint8_t *stage_all, int threads) {
  int st = check_params(p);
  if (st) return st;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!isfinite(xyz[i])) return ORC_ENONFINITE;
  if (o->n_leaves) *o->n_leaves = 0;
  if (n == 0) return ORC_OK;

  /* R1: root cube */
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) { lo[a] = xyz[a]; hi[a] = xyz[a]; }
  for (int64_t i = 1; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      float v = xyz[3 * i + a];
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
  float side = 0.0f;
  for (int a = 0; a < 3; ++a) {
    float e = hi[a] - lo[a];
    if (e > side) side = e;
  }
  if (side == 0.0f) side = 1.0f;
  float s = 2097152.0f / side;
  if (o->root) { o->root[0] = lo[0]; o->root[1] = lo[1]; o->root[2] = lo[2]; o->root[3] = side; }

  keyed_t *sorted = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)n);
  leaf_t *leaves = (leaf_t *)malloc(sizeof(leaf_t) * (size_t)n);
  if (!sorted || !leaves) return ORC_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) q[a] = quantise(xyz[3 * i + a], lo[a], s);
    sorted[i].key = orc_interleave(q[0], q[1], q[2]);
    sorted[i].idx = (uint32_t)i;
    if (o->key) o->key[i] = sorted[i].key;
  }
  /* Sec. 3: sort by (key, index), then split top-down (R2) */
  qsort(sorted, (size_t)n, sizeof(keyed_t), cmp_keyed);
  octree_t tree = {sorted, p->leaf_capacity, p->max_depth, leaves, 0};
  octree_build(&tree, 0, 0, (uint32_t)n);
  if (o->n_leaves) *o->n_leaves = tree.n_leaves;

  ctx_t c = {xyz, p, side * INV_TWO21, o, dF, F_all, stage_all};
  for (int64_t i = 0; i < n; ++i) { F_all[i] = 0.0; stage_all[i] = 0; }
  /* The leaves are independent (each writes only its own points' entries), so
   * with threads > 1 they are spread over threads; the arithmetic of every leaf
   * is the same either way.  (Used only to time the oracle on all host cores.) */
  if (p->cross_leaf) {  /* R14 */
    for (int64_t L = 0; L < tree.n_leaves; ++L) {
      if (o->leaf_start) o->leaf_start[L] = leaves[L].start;
      if (o->leaf_count) o->leaf_count[L] = leaves[L].count;
      if (o->leaf_level) o->leaf_level[L] = leaves[L].level;
    }
    st = run_cross_leaf(&c, sorted, n, leaves, tree.n_leaves);
  }
  int failed = 0;
  if (!p->cross_leaf) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
  for (int64_t L = 0; L < tree.n_leaves; ++L) {
    if (o->leaf_start) o->leaf_start[L] = leaves[L].start;
    if (o->leaf_count) o->leaf_count[L] = leaves[L].count;
    if (o->leaf_level) o->leaf_level[L] = leaves[L].level;
    if (process_leaf(&c, sorted, &leaves[L], (uint32_t)L) != ORC_OK) failed = 1;
  }
  }
  if (failed) st = ORC_ENOMEM;
  /* Eq. 22: the union of the leaves' survivors, as a mask in input order */
  for (int64_t i = 0; i < n; ++i) {
    if (o->stage) o->stage[i] = stage_all[i];
    if (o->mask) o->mask[i] = stage_all[i] == 0;
    if (o->score) o->score[i] = F_all[i];
  }
  free(sorted);
  free(leaves);
  return st;
}

int orc_denoise(const float *xyz, int64_t n, const orc_params *p, orc_out *out) {
  return orc_denoise_threads(xyz, n, p, out, 1);
}

int orc_denoise_threads(const float *xyz, int64_t n, const orc_params *p, orc_out *out, int threads) {
  orc_out none;
  memset(&none, 0, sizeof none);
  if (!out) out = &none;
  double *F = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  uint8_t *stg = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
  if (!F || !stg) return ORC_ENOMEM;
  int st = run(xyz, n, p, out, NULL, F, stg, threads);
  free(F);
  free(stg);
  return st;
}

/* R12: soft-F1 of the differentiable form and its exact gradient */
int orc_softf1(const float *xyz, int64_t n, const orc_params *p, const uint8_t *noise,
               const uint8_t *in_loss, double *loss, double grad[4], double *removal) {
  orc_out none;
  memset(&none, 0, sizeof none);
  size_t nn = (size_t)(n > 0 ? n : 1);
  double *F = (double *)malloc(sizeof(double) * nn);
  double *dF = (double *)malloc(sizeof(double) * nn * 3);
  double *rm = (double *)malloc(sizeof(double) * nn);
  double *dm = (double *)malloc(sizeof(double) * nn);   /* m(1-m)/T on P_2 */
  uint8_t *stg = (uint8_t *)malloc(nn);
  if (!F || !dF || !rm || !dm || !stg) return ORC_ENOMEM;
  orc_params q = *p;
  q.select_mode = 1;
  int st = run(xyz, n, &q, &none, dF, F, stg, 1);
  if (st) return st;
  const double T = p->temperature, tau = p->tau;
  double Sr = 0.0, Sy = 0.0, Sry = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int scored = (stg[i] == 0 || stg[i] == 3);
    double m = 0.0;
    dm[i] = 0.0;
    if (scored && F[i] > 0.0) {
      double z = (log(F[i]) - tau) / T;
      m = 1.0 / (1.0 + exp(-z));
      dm[i] = m * (1.0 - m) / T;
    }
    rm[i] = 1.0 - m;
    if (removal) removal[i] = rm[i];
    if (in_loss && !in_loss[i]) continue;
    Sr += rm[i];
    Sy += (double)noise[i];
    Sry += rm[i] * (double)noise[i];
  }
  double den = Sr + Sy;
  *loss = (den > 0.0) ? 1.0 - 2.0 * Sry / den : 1.0;
  double g[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n && den > 0.0; ++i) {
    if (in_loss && !in_loss[i]) continue;
    if (dm[i] == 0.0) continue;
    /* d loss / d r_i */
    double dl_dr = -2.0 * ((double)noise[i] * den - Sry) / (den * den);
    /* r_i = 1 - sigmoid((ln F - tau)/T):  dr/dF = -m(1-m)/(T F), dr/dtau = m(1-m)/T */
    double dr_dF = -dm[i] / F[i];
    for (int k = 0; k < 3; ++k) g[k] += dl_dr * dr_dF * dF[3 * i + k];
    g[3] += dl_dr * dm[i];
  }
  for (int k = 0; k < 4; ++k) grad[k] = g[k];
  free(F); free(dF); free(rm); free(dm); free(stg);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Eq. 29-30: nearest-neighbour distances, Chamfer distance and PSNR    */
/* ------------------------------------------------------------------ */
int orc_nn_d2(const float *a, int64_t na, const float *b, int64_t nb, double *out) {
  if (na < 0 || nb <= 0 || !out) return ORC_EINVAL;
  for (int64_t i = 0; i < na; ++i) {
    double best = INFINITY;
    for (int64_t j = 0; j < nb; ++j) {
      double d2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        double t = (double)a[3 * i + c] - (double)b[3 * j + c];
        d2 += t * t;
      }
      if (d2 < best) best = d2;
    }
    out[i] = best;
  }
  return ORC_OK;
}

int orc_metrics(const float *clean, int64_t na, const float *den, int64_t nb, double *mse, double *cd,
                double *psnr) {
  if (na <= 0 || nb <= 0) return ORC_EINVAL;
  double *da = (double *)malloc(sizeof(double) * (size_t)na);
  double *db = (double *)malloc(sizeof(double) * (size_t)nb);
  if (!da || !db) return ORC_ENOMEM;
  orc_nn_d2(clean, na, den, nb, da);
  orc_nn_d2(den, nb, clean, na, db);
  double sa = 0.0, sb = 0.0;
  for (int64_t i = 0; i < na; ++i) sa += da[i];
  for (int64_t j = 0; j < nb; ++j) sb += db[j];
  const double m = sa / (double)na;
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) lo[c] = hi[c] = clean[c];
  for (int64_t i = 1; i < na; ++i)
    for (int c = 0; c < 3; ++c) {
      if (clean[3 * i + c] < lo[c]) lo[c] = clean[3 * i + c];
      if (clean[3 * i + c] > hi[c]) hi[c] = clean[3 * i + c];
    }
  double M2 = 0.0;
  for (int c = 0; c < 3; ++c) M2 += (hi[c] - lo[c]) * (hi[c] - lo[c]);
  if (mse) *mse = m;
  if (cd) *cd = m + sb / (double)nb;
  if (psnr) *psnr = 10.0 * log10(M2 / m);
  free(da);
  free(db);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2, Eq. 1-9: the gravitational-function baseline               */
/* ------------------------------------------------------------------ */
int orc_baseline(const float *xyz, int64_t n, double G, double alpha, uint8_t *keep, uint32_t *n_i,
                 double *d_i, double *F_i, double *R_out, double *T_out) {
  if (n <= 0 || !keep) return ORC_EINVAL;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!isfinite(xyz[i])) return ORC_ENONFINITE;
  /* Eq. 1: centroid */
  double theta[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) theta[c] += (double)xyz[3 * i + c];
  for (int c = 0; c < 3; ++c) theta[c] /= (double)n;
  /* Eq. 2: extents */
  double H[3];
  for (int c = 0; c < 3; ++c) {
    float lo = xyz[c], hi = xyz[c];
    for (int64_t i = 1; i < n; ++i) {
      if (xyz[3 * i + c] < lo) lo = xyz[3 * i + c];
      if (xyz[3 * i + c] > hi) hi = xyz[3 * i + c];
    }
    H[c] = (double)hi - (double)lo;
  }
  /* Eq. 3: neighbourhood radius; Eq. 7: threshold */
  const double R = 6.0 * (H[0] * H[1] + H[0] * H[2] + H[1] * H[2]) / (double)n;
  const double T = alpha * G * (H[0] + H[1] + H[2]) / (double)n;
  const double R2 = R * R;
  if (R_out) *R_out = R;
  if (T_out) *T_out = T;
  for (int64_t i = 0; i < n; ++i) {
    /* Eq. 4 */
    double dd = 0.0;
    for (int c = 0; c < 3; ++c) {
      double t = (double)xyz[3 * i + c] - theta[c];
      dd += t * t;
    }
    const double d = sqrt(dd);
    /* Eq. 5: every point within R, the point itself included */
    uint32_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
      float dx = xyz[3 * j] - xyz[3 * i];
      float dy = xyz[3 * j + 1] - xyz[3 * i + 1];
      float dz = xyz[3 * j + 2] - xyz[3 * i + 2];
      float xx = dx * dx;
      float d2 = fmaf(dz, dz, fmaf(dy, dy, xx));
      cnt += ((double)d2 <= R2);
    }
    /* Eq. 6 and Eq. 8 */
    const double F = G * (double)cnt / (d * d);
    keep[i] = F >= T / d;
    if (n_i) n_i[i] = cnt;
    if (d_i) d_i[i] = d;
    if (F_i) F_i[i] = F;
  }
  return ORC_OK;
}

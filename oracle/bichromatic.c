/*
 * bichromatic.c -- FP64 oracle of the bichromatic case (test
 * infrastructure; only tests/, smoke() and the bench's CPU legs use it).
 *
 * Outlook of Schubert & Rousseeuw, "Fast and Eager k-Medoids Clustering"
 * (arXiv 2008.05171): possible locations L and consumers C are different
 * sets, the medoids are chosen among the locations, and the bichromatic
 * medoid of the consumers is medoid(L, C) = argmin_{x_l in L} sum_{x_c in C}
 * d(x_c, x_l).  The objective is Eq. (2) summed over the consumers, TD =
 * sum_{x_c in C} min_j d(x_c, m_j); BUILD (Alg. 1) adds the location whose
 * addition lowers TD the most; FastPAM1 (Alg. 3, Eq. (7)) evaluates every
 * (medoid slot, non-medoid location) swap with the removal loss, the shared
 * term and the per-slot corrections accumulated over the consumers.  The
 * paper gives no further detail for this case: every step is the square
 * case's with the candidate loop over L and the point loop over C.
 *
 * Matrix: m rows (locations) of ld elements, d(x_c, x_l) = D[l * ld + c]
 * for consumer c in [0, n); dtype 0 = int32, 1 = float32.  Ties: lowest
 * slot, then lowest location index (as the square oracle).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BI_INF (1.0 / 0.0)

static double bd(const void *D, int dtype, int64_t ld, int64_t l, int64_t c) {
  size_t idx = (size_t)l * (size_t)ld + (size_t)c;
  if (dtype == 0) return (double)((const int32_t *)D)[idx];
  return (double)((const float *)D)[idx];
}

/* TD over the consumers, Eq. (2); labels[c] = lowest nearest slot. */
double oracle_bi_td(const void *D, int dtype, int64_t m, int64_t n, int64_t ld,
                    const int32_t *med, int k, int32_t *labels) {
  (void)m;
  double td = 0.0;
  for (int64_t c = 0; c < n; c++) {
    double best = BI_INF;
    int lab = -1;
    for (int j = 0; j < k; j++) {
      double v = bd(D, dtype, ld, med[j], c);
      if (v < best) {
        best = v;
        lab = j;
      }
    }
    td += best;
    if (labels) labels[c] = lab;
  }
  return td;
}

/* Nearest / second-nearest slot of every consumer (Sec. 2), k = 1: sec = -1,
 * d_s = +inf. */
static void bi_cache(const void *D, int dtype, int64_t n, int64_t ld,
                     const int32_t *med, int k, int32_t *near, double *dn,
                     double *ds) {
  for (int64_t c = 0; c < n; c++) {
    int n1 = -1;
    double d1 = BI_INF, d2 = BI_INF;
    for (int j = 0; j < k; j++) {
      double v = bd(D, dtype, ld, med[j], c);
      if (v < d1) {
        d2 = d1;
        n1 = j;
        d1 = v;
      } else if (v < d2) {
        d2 = v;
      }
    }
    near[c] = n1;
    dn[c] = d1;
    ds[c] = d2;
  }
}

/* BUILD (Alg. 1) over the locations: step 0 takes the bichromatic medoid of
 * the consumers, each later step the location with the least
 * sum_c min(d(x_c, x_l) - d_n(x_c), 0).  step_delta[0] = the first
 * location's distance sum, step_delta[t] = the gain of step t. */
int oracle_bi_build(const void *D, int dtype, int64_t m, int64_t n, int64_t ld,
                    int k, int32_t *med, double *td_out, double *step_delta) {
  if (m <= 0 || n <= 0 || k <= 0 || k > m) return -1;
  double *dnear = (double *)malloc(sizeof(double) * (size_t)n);
  char *is_med = (char *)calloc((size_t)m, 1);
  double td = 0.0;
  for (int t = 0; t < k; t++) {
    double best = BI_INF;
    int64_t bl = -1;
    for (int64_t l = 0; l < m; l++) {
      if (is_med[l]) continue;
      double g = 0.0;
      for (int64_t c = 0; c < n; c++) {
        double v = bd(D, dtype, ld, l, c);
        if (t == 0) {
          g += v;
        } else {
          double dd = v - dnear[c];
          if (dd < 0.0) g += dd;
        }
      }
      if (g < best) {
        best = g;
        bl = l;
      }
    }
    if (bl < 0) /* only reachable with NaN input: lowest free location */
      for (bl = 0; is_med[bl]; bl++) {
      }
    med[t] = (int32_t)bl;
    is_med[bl] = 1;
    td = (t == 0) ? best : td + best;
    if (step_delta) step_delta[t] = best;
    for (int64_t c = 0; c < n; c++) {
      double v = bd(D, dtype, ld, bl, c);
      if (t == 0 || v < dnear[c]) dnear[c] = v;
    }
  }
  if (td_out) *td_out = td;
  free(dnear);
  free(is_med);
  return 0;
}

/* One evaluation of every swap (slot i, non-medoid location l).
 * cand_delta[l] = min_i Delta(i, l), cand_slot[l] its lowest slot (+inf and
 * -1 for medoids); the best (Delta, slot, location) in lexicographic order.
 * method 0: brute force, TD of the swapped set recomputed by Eq. (2);
 * method 2: FastPAM1, Eq. (7) over the consumers (k >= 2). */
void oracle_bi_eval_swaps(const void *D, int dtype, int64_t m, int64_t n,
                          int64_t ld, const int32_t *med, int k, int method,
                          double *cand_delta, int32_t *cand_slot,
                          double *best_delta, int32_t *best_slot,
                          int64_t *best_cand) {
  char *is_med = (char *)calloc((size_t)m, 1);
  for (int j = 0; j < k; j++) is_med[med[j]] = 1;
  int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  double *ds = (double *)malloc(sizeof(double) * (size_t)n);
  double *rl = (double *)malloc(sizeof(double) * (size_t)k);
  bi_cache(D, dtype, n, ld, med, k, near, dn, ds);
  /* removal loss, Eq. (7): Delta^{-m_i} = sum_{nearest(c) = i} (d_s - d_n) */
  for (int i = 0; i < k; i++) rl[i] = 0.0;
  for (int64_t c = 0; c < n; c++) rl[near[c]] += ds[c] - dn[c];
  const double td0 = (method == 0) ? oracle_bi_td(D, dtype, m, n, ld, med, k, NULL) : 0.0;
#pragma omp parallel
  {
    double *acc = (double *)malloc(sizeof(double) * (size_t)k);
    int32_t *trial = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
#pragma omp for schedule(dynamic, 16)
    for (int64_t l = 0; l < m; l++) {
      if (is_med[l]) {
        cand_delta[l] = BI_INF;
        cand_slot[l] = -1;
        continue;
      }
      if (method == 0) {
        for (int i = 0; i < k; i++) {
          memcpy(trial, med, sizeof(int32_t) * (size_t)k);
          trial[i] = (int32_t)l;
          acc[i] = oracle_bi_td(D, dtype, m, n, ld, trial, k, NULL) - td0;
        }
      } else {
        for (int i = 0; i < k; i++) acc[i] = rl[i];
        double plus = 0.0; /* shared term Delta^{+x_l} */
        for (int64_t c = 0; c < n; c++) {
          double v = bd(D, dtype, ld, l, c);
          if (v < dn[c]) { /* x_l becomes the nearest medoid of x_c */
            plus += v - dn[c];
            acc[near[c]] += dn[c] - ds[c];
          } else if (v < ds[c]) { /* x_l would be the second nearest */
            acc[near[c]] += v - ds[c];
          }
        }
        for (int i = 0; i < k; i++) acc[i] += plus;
      }
      int bi = 0;
      for (int i = 1; i < k; i++)
        if (acc[i] < acc[bi]) bi = i;
      cand_delta[l] = acc[bi];
      cand_slot[l] = bi;
    }
    free(acc);
    free(trial);
  }
  /* the least (Delta, slot, location) */
  *best_delta = BI_INF;
  *best_slot = -1;
  *best_cand = -1;
  for (int64_t l = 0; l < m; l++) {
    if (is_med[l]) continue;
    if (cand_delta[l] < *best_delta ||
        (cand_delta[l] == *best_delta && cand_slot[l] < *best_slot)) {
      *best_delta = cand_delta[l];
      *best_slot = cand_slot[l];
      *best_cand = l;
    }
  }
  free(is_med);
  free(near);
  free(dn);
  free(ds);
  free(rl);
}

/* FastPAM1 SWAP to convergence (Alg. 3) from the given medoids: each pass
 * applies the best swap iff its Delta < -tol.  k = 1: the best single swap
 * is the location with the least distance sum (the bichromatic medoid).
 * stats[0] = passes, stats[1] = swaps, stats[2] = converged.  td[0] = TD
 * bookkept as TD + Delta*, td[1] = TD recomputed.  The trace records
 * (Delta, slot, location) of every applied swap up to cap. */
int oracle_bi_swap(const void *D, int dtype, int64_t m, int64_t n, int64_t ld,
                   int k, int32_t *med, int max_iter, double tol,
                   int64_t *stats, double *td, int trace_cap, double *tr_d,
                   int32_t *tr_i, int64_t *tr_c) {
  if (m <= 0 || n <= 0 || k <= 0 || k > m) return -1;
  double *cd = (double *)malloc(sizeof(double) * (size_t)m);
  int32_t *cs = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
  double book = oracle_bi_td(D, dtype, m, n, ld, med, k, NULL);
  int64_t iters = 0, swaps = 0, conv = 0;
  while (iters < max_iter) {
    double bdlt;
    int32_t bslot;
    int64_t bcand;
    iters++;
    if (k == 1) {
      double s0 = 0.0;
      for (int64_t c = 0; c < n; c++) s0 += bd(D, dtype, ld, med[0], c);
      bdlt = BI_INF;
      bslot = 0;
      bcand = -1;
      for (int64_t l = 0; l < m; l++) {
        if (l == med[0]) continue;
        double s = 0.0;
        for (int64_t c = 0; c < n; c++) s += bd(D, dtype, ld, l, c);
        if (s - s0 < bdlt) {
          bdlt = s - s0;
          bcand = l;
        }
      }
    } else {
      oracle_bi_eval_swaps(D, dtype, m, n, ld, med, k, 2, cd, cs, &bdlt, &bslot,
                           &bcand);
    }
    if (bcand < 0 || !(bdlt < -tol)) {
      conv = 1;
      break;
    }
    if (swaps < trace_cap) {
      if (tr_d) tr_d[swaps] = bdlt;
      if (tr_i) tr_i[swaps] = bslot;
      if (tr_c) tr_c[swaps] = bcand;
    }
    med[bslot] = (int32_t)bcand;
    book += bdlt;
    swaps++;
  }
  stats[0] = iters;
  stats[1] = swaps;
  stats[2] = conv;
  td[0] = book;
  td[1] = oracle_bi_td(D, dtype, m, n, ld, med, k, NULL);
  free(cd);
  free(cs);
  return 0;
}

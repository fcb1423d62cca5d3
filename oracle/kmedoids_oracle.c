/*
 * kmedoids_oracle.c -- the ORACLE for the k-medoids hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, deliberately obvious FP64 CPU
 * implementation of what the paper (Schubert & Rousseeuw, "Fast and Eager
 * k-Medoids Clustering", arXiv 2008.05171) computes: the TD objective, PAM
 * BUILD, PAM SWAP (by brute-force TD recomputation and by the cached change
 * function), FastPAM1, FastPAM2, FasterPAM and CLARA.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load this
 * file; the product path (the CUDA library) never does, and the two share no
 * code, header, table or helper.
 *
 * Conventions (every function):
 *   D      n x n dissimilarities, row-major with row stride ld (elements);
 *          dtype 0 = int32, 1 = float32.  d(o,c) := D[o*ld + c], read as an
 *          FP64 value.  D is assumed symmetric with a zero diagonal and
 *          finite non-negative entries (the paper's symmetric special case,
 *          Sec. 1.2); asymmetric input is out of scope.
 *   med    k medoid point indices in slot order; a swap keeps the slot
 *          ("swap roles", Alg. 2 / Alg. 3).
 *   All sums are FP64 (exact for int32 data while |TD| < 2^53).
 *
 * Tie rules (the paper only fixes "prefer the smaller index i on ties",
 * Sec. 3.1, and strict comparisons in its listings): nearest medoid = lowest
 * slot among equal distances; per-candidate slot = lowest slot; global swap =
 * lexicographic minimum of (delta, slot, candidate); BUILD = lowest point
 * index among equal gains.
 *
 * Parity status: every function below is pinned by tests (worked example of
 * Fig. 1, brute-force TD differences, exhaustive case tables, enumeration of
 * all medoid sets on tiny inputs, invariants).  FastPAM2's additional swaps
 * are pinned to a brute-force replay of the reading stated at the function,
 * but the reading itself is "parity unpinned": the paper describes FastPAM2
 * only in words (Sec. 3.2) and prints no values for it.  CLARA's sample
 * quality is "parity unpinned" beyond the invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_INF (1.0 / 0.0)

typedef struct {
  const void *D;
  int dtype;
  int64_t n;
  int64_t ld;
} or_mat;

/* d(x_o, x_c) as an FP64 value. */
static double od(const or_mat *m, int64_t o, int64_t c) {
  size_t idx = (size_t)o * (size_t)m->ld + (size_t)c;
  if (m->dtype == 0) return (double)((const int32_t *)m->D)[idx];
  return (double)((const float *)m->D)[idx];
}

static or_mat mk(const void *D, int dtype, int64_t n, int64_t ld) {
  or_mat m;
  m.D = D;
  m.dtype = dtype;
  m.n = n;
  m.ld = ld;
  return m;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------
 * TD objective, Eq. (2) "eqn:td": TD = sum_o min_j d(o, m_j).
 * labels[o] = lowest slot attaining the minimum (may be NULL).
 * ---------------------------------------------------------------------- */
double oracle_td(const void *D, int dtype, int64_t n, int64_t ld,
                 const int32_t *med, int k, int32_t *labels) {
  or_mat m = mk(D, dtype, n, ld);
  double td = 0.0;
  for (int64_t o = 0; o < n; o++) {
    double best = OR_INF;
    int lab = -1;
    for (int j = 0; j < k; j++) {
      double v = od(&m, o, med[j]);
      if (v < best) {
        best = v;
        lab = j;
      }
    }
    td += best;
    if (labels) labels[o] = lab;
  }
  return td;
}

/* ------------------------------------------------------------------------
 * Per-point cache (Sec. 2, "nearest(o), d_n(o), d_s(o)"; Alg. 2 and 3):
 * nearest slot, its distance, second-nearest slot and its distance, taken
 * as the two smallest (distance, slot) pairs in lexicographic order.
 * k = 1: sec = -1, d_s = +inf.
 * ---------------------------------------------------------------------- */
void oracle_cache(const void *D, int dtype, int64_t n, int64_t ld,
                  const int32_t *med, int k, int32_t *near, int32_t *sec,
                  double *dn, double *ds) {
  or_mat m = mk(D, dtype, n, ld);
  for (int64_t o = 0; o < n; o++) {
    int n1 = -1, n2 = -1;
    double d1 = OR_INF, d2 = OR_INF;
    for (int j = 0; j < k; j++) {
      double v = od(&m, o, med[j]);
      if (v < d1) {
        n2 = n1;
        d2 = d1;
        n1 = j;
        d1 = v;
      } else if (v < d2) {
        n2 = j;
        d2 = v;
      }
    }
    near[o] = n1;
    if (sec) sec[o] = n2;
    dn[o] = d1;
    ds[o] = d2;
  }
}

/* Removal loss, Eq. (7) first line: Delta^{-m_i} = sum_{nearest(o)=i}
 * (d_s(o) - d_n(o)), for all slots in one pass over the points. */
void oracle_removal_loss(int64_t n, int k, const int32_t *near,
                         const double *dn, const double *ds, double *rl) {
  for (int i = 0; i < k; i++) rl[i] = 0.0;
  for (int64_t o = 0; o < n; o++) rl[near[o]] += ds[o] - dn[o];
}

/* ------------------------------------------------------------------------
 * PAM BUILD, Alg. 1, read with the self term included (the gain of adding
 * x_c counts o = c, so each step's gain is the exact TD change and the
 * bookkept TD equals Eq. (2)).  step_delta[0] = first medoid's distance sum,
 * step_delta[i] = gain of step i (may be NULL).  Returns 0.
 * ---------------------------------------------------------------------- */
int oracle_build(const void *D, int dtype, int64_t n, int64_t ld, int k,
                 int32_t *med, double *td_out, double *step_delta) {
  if (n <= 0 || k <= 0 || k > n) return -1;
  or_mat m = mk(D, dtype, n, ld);
  double *dnear = (double *)malloc(sizeof(double) * (size_t)n);
  char *is_med = (char *)calloc((size_t)n, 1);
  double *gain = (double *)malloc(sizeof(double) * (size_t)n);

  /* First medoid: smallest distance sum (Eq. (3), the 1-medoid). */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; c++) {
    double s = 0.0;
    for (int64_t o = 0; o < n; o++) s += od(&m, o, c);
    gain[c] = s;
  }
  double td = OR_INF;
  int64_t m1 = -1;
  for (int64_t c = 0; c < n; c++)
    if (gain[c] < td) {
      td = gain[c];
      m1 = c;
    }
  if (m1 < 0) m1 = 0; /* only reachable with NaN input */
  med[0] = (int32_t)m1;
  is_med[m1] = 1;
  if (step_delta) step_delta[0] = td;
  for (int64_t o = 0; o < n; o++) dnear[o] = od(&m, o, m1);

  /* Remaining medoids: add the point whose addition lowers TD the most. */
  for (int i = 1; i < k; i++) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) {
      if (is_med[c]) continue;
      double delta = 0.0;
      for (int64_t o = 0; o < n; o++) {
        double dd = od(&m, o, c) - dnear[o];
        if (dd < 0.0) delta += dd;
      }
      gain[c] = delta;
    }
    double best = OR_INF;
    int64_t bc = -1;
    for (int64_t c = 0; c < n; c++)
      if (!is_med[c] && gain[c] < best) {
        best = gain[c];
        bc = c;
      }
    if (bc < 0) /* only reachable with NaN input: lowest non-medoid */
      for (bc = 0; is_med[bc]; bc++) {
      }
    med[i] = (int32_t)bc;
    is_med[bc] = 1;
    td += best;
    if (step_delta) step_delta[i] = best;
    for (int64_t o = 0; o < n; o++) {
      double v = od(&m, o, bc);
      if (v < dnear[o]) dnear[o] = v;
    }
  }
  if (td_out) *td_out = td;
  free(dnear);
  free(is_med);
  free(gain);
  return 0;
}

/* One BUILD step of Alg. 1 given the medoids chosen so far (t of them):
 * gains[c] = sum_o min(d(o,c) - d_n(o), 0) for non-medoids (t > 0), or the
 * distance sum of c (t = 0); medoids get +inf. */
void oracle_build_gains(const void *D, int dtype, int64_t n, int64_t ld,
                        const int32_t *med, int t, double *gains) {
  or_mat m = mk(D, dtype, n, ld);
  double *dnear = (double *)malloc(sizeof(double) * (size_t)n);
  char *is_med = (char *)calloc((size_t)n, 1);
  for (int j = 0; j < t; j++) is_med[med[j]] = 1;
  for (int64_t o = 0; o < n; o++) {
    double b = OR_INF;
    for (int j = 0; j < t; j++) {
      double v = od(&m, o, med[j]);
      if (v < b) b = v;
    }
    dnear[o] = b;
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; c++) {
    if (is_med[c]) {
      gains[c] = OR_INF;
      continue;
    }
    double g = 0.0;
    for (int64_t o = 0; o < n; o++) {
      if (t == 0) {
        g += od(&m, o, c);
      } else {
        double dd = od(&m, o, c) - dnear[o];
        if (dd < 0.0) g += dd;
      }
    }
    gains[c] = g;
  }
  free(dnear);
  free(is_med);
}

/* ------------------------------------------------------------------------
 * One evaluation of all swaps (medoid slot i, non-medoid candidate c).
 * Outputs, per point c: cand_delta[c] = min_i Delta(i,c) and cand_slot[c] =
 * the lowest slot attaining it (+inf / -1 for medoids), plus the global
 * lexicographic minimum of (Delta, i, c).
 *
 * method 0: brute force, Delta(i,c) = TD(M - m_i + c) - TD(M) by full
 *           recomputation of Eq. (2) (tiny n only).
 * method 1: PAM, Alg. 2 with the cached change function of Eq. (5).
 * method 2: FastPAM1, Alg. 3 with the decomposition of Eq. (7): removal
 *           loss + shared accumulator Delta^{+x_c} + per-slot corrections.
 * ---------------------------------------------------------------------- */
typedef struct {
  double delta;
  int slot;
  int64_t cand;
} or_key;

static int key_less(double d, int i, int64_t c, const or_key *b) {
  if (d != b->delta) return d < b->delta;
  if (i != b->slot) return i < b->slot;
  return c < b->cand;
}

/* Eq. (5): change of TD contributed by x_o when slot i is replaced by x_c. */
static double change_eq5(double doc, int near_o, double dn_o, double ds_o,
                         int i) {
  if (near_o != i) {
    if (doc >= dn_o) return 0.0;  /* (a) */
    return doc - dn_o;            /* (c) */
  }
  if (doc < ds_o) return doc - dn_o; /* (b1) */
  return ds_o - dn_o;                /* (b2) */
}

static void eval_all(const or_mat *m, const int32_t *med, int k, int method,
                     double *cand_delta, int32_t *cand_slot, or_key *best) {
  int64_t n = m->n;
  char *is_med = (char *)calloc((size_t)n, 1);
  for (int j = 0; j < k; j++) is_med[med[j]] = 1;
  int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  double *ds = (double *)malloc(sizeof(double) * (size_t)n);
  double *rl = (double *)malloc(sizeof(double) * (size_t)k);
  oracle_cache(m->D, m->dtype, n, m->ld, med, k, near, NULL, dn, ds);
  oracle_removal_loss(n, k, near, dn, ds, rl);
  double td0 = 0.0;
  if (method == 0) td0 = oracle_td(m->D, m->dtype, n, m->ld, med, k, NULL);

#pragma omp parallel
  {
    double *acc = (double *)malloc(sizeof(double) * (size_t)k);
    int32_t *trial = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
#pragma omp for schedule(dynamic, 16)
    for (int64_t c = 0; c < n; c++) {
      if (is_med[c]) {
        cand_delta[c] = OR_INF;
        cand_slot[c] = -1;
        continue;
      }
      if (method == 0) {
        for (int i = 0; i < k; i++) {
          memcpy(trial, med, sizeof(int32_t) * (size_t)k);
          trial[i] = (int32_t)c;
          acc[i] = oracle_td(m->D, m->dtype, n, m->ld, trial, k, NULL) - td0;
        }
      } else if (method == 1) {
        for (int i = 0; i < k; i++) {
          double s = 0.0;
          for (int64_t o = 0; o < n; o++)
            s += change_eq5(od(m, o, c), near[o], dn[o], ds[o], i);
          acc[i] = s;
        }
      } else {
        double plus = 0.0; /* shared accumulator Delta^{+x_c} */
        for (int i = 0; i < k; i++) acc[i] = rl[i];
        for (int64_t o = 0; o < n; o++) {
          double doc = od(m, o, c);
          if (doc < dn[o]) { /* x_c becomes the nearest medoid of x_o */
            plus += doc - dn[o];
            acc[near[o]] += dn[o] - ds[o];
          } else if (doc < ds[o]) { /* x_c would be the second nearest */
            acc[near[o]] += doc - ds[o];
          }
        }
        for (int i = 0; i < k; i++) acc[i] += plus;
      }
      int bi = 0;
      for (int i = 1; i < k; i++)
        if (acc[i] < acc[bi]) bi = i;
      cand_delta[c] = acc[bi];
      cand_slot[c] = bi;
    }
    free(acc);
    free(trial);
  }
  best->delta = OR_INF;
  best->slot = -1;
  best->cand = -1;
  for (int64_t c = 0; c < n; c++)
    if (!is_med[c] && key_less(cand_delta[c], cand_slot[c], c, best)) {
      best->delta = cand_delta[c];
      best->slot = cand_slot[c];
      best->cand = c;
    }
  free(is_med);
  free(near);
  free(dn);
  free(ds);
  free(rl);
}

void oracle_eval_swaps(const void *D, int dtype, int64_t n, int64_t ld,
                       const int32_t *med, int k, int method,
                       double *cand_delta, int32_t *cand_slot,
                       double *best_delta, int32_t *best_slot,
                       int64_t *best_cand) {
  or_mat m = mk(D, dtype, n, ld);
  or_key b;
  eval_all(&m, med, k, method, cand_delta, cand_slot, &b);
  *best_delta = b.delta;
  *best_slot = b.slot;
  *best_cand = b.cand;
}

/* Delta of one swap (slot i -> point c) by Eq. (4)/(5) summed over all
 * points with a fresh cache.  Points that are other medoids contribute 0
 * under Eq. (5), so summing over every x_o equals the listing's sum. */
double oracle_swap_delta(const void *D, int dtype, int64_t n, int64_t ld,
                         const int32_t *med, int k, int slot, int64_t c) {
  or_mat m = mk(D, dtype, n, ld);
  int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  double *ds = (double *)malloc(sizeof(double) * (size_t)n);
  oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
  double s = 0.0;
  for (int64_t o = 0; o < n; o++)
    s += change_eq5(od(&m, o, c), near[o], dn[o], ds[o], slot);
  free(near);
  free(dn);
  free(ds);
  return s;
}

/* ------------------------------------------------------------------------
 * k = 1: d_s is undefined, so the decomposition does not apply.  The best
 * single swap is the 1-medoid of Eq. (3) (smallest distance sum, lowest
 * index on ties); swap to it iff it lowers TD.
 * ---------------------------------------------------------------------- */
static void one_medoid_eval(const or_mat *m, const int32_t *med, or_key *b) {
  int64_t n = m->n;
  double *s = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; c++) {
    double t = 0.0;
    for (int64_t o = 0; o < n; o++) t += od(m, o, c);
    s[c] = t;
  }
  b->delta = OR_INF;
  b->slot = 0;
  b->cand = -1;
  for (int64_t c = 0; c < n; c++)
    if (c != med[0] && s[c] - s[med[0]] < b->delta) {
      b->delta = s[c] - s[med[0]];
      b->cand = c;
    }
  free(s);
}

/* ------------------------------------------------------------------------
 * SWAP loops.
 *   variant 0: PAM, brute-force deltas      (Alg. 2, Eq. (2) recomputed)
 *   variant 1: PAM, cached change function  (Alg. 2, Eq. (5))
 *   variant 2: FastPAM1                     (Alg. 3, Eq. (7))
 *   variant 3: FastPAM2                     (Sec. 3.2, read as below)
 *   variant 4: FasterPAM                    (Alg. 4, read as below)
 * stats[0] = iterations, stats[1] = swaps, stats[2] = converged (1) or
 * stopped by max_iter (0), stats[3] = positions visited (FasterPAM only).
 * td[0] = TD bookkept as TD + Delta*, td[1] = TD recomputed by Eq. (2).
 * The trace records every applied swap (delta, slot, candidate) up to cap.
 * ---------------------------------------------------------------------- */
static void apply_trace(int64_t *nt, int cap, double *tr_d, int32_t *tr_i,
                        int64_t *tr_c, double d, int i, int64_t c) {
  if (*nt < cap) {
    if (tr_d) tr_d[*nt] = d;
    if (tr_i) tr_i[*nt] = i;
    if (tr_c) tr_c[*nt] = c;
  }
  (*nt)++;
}

/* FastPAM1 delta of one candidate against the current cache: returns
 * min_i Delta(i, c) and its lowest slot (Eq. (7)). */
static double fastpam1_candidate(const or_mat *m, int k, const int32_t *near,
                                 const double *dn, const double *ds,
                                 const double *rl, int64_t c, double *acc,
                                 int *slot) {
  double plus = 0.0;
  for (int i = 0; i < k; i++) acc[i] = rl[i];
  for (int64_t o = 0; o < m->n; o++) {
    double doc = od(m, o, c);
    if (doc < dn[o]) {
      plus += doc - dn[o];
      acc[near[o]] += dn[o] - ds[o];
    } else if (doc < ds[o]) {
      acc[near[o]] += doc - ds[o];
    }
  }
  int bi = 0;
  for (int i = 1; i < k; i++)
    if (acc[i] < acc[bi]) bi = i;
  *slot = bi;
  return acc[bi] + plus;
}

int oracle_swap(const void *D, int dtype, int64_t n, int64_t ld, int k,
                int32_t *med, int variant, int max_iter, double tol,
                double fp2_tol, int64_t *stats, double *td, int trace_cap,
                double *tr_d, int32_t *tr_i, int64_t *tr_c) {
  or_mat m = mk(D, dtype, n, ld);
  int64_t iters = 0, swaps = 0, conv = 0, visited = 0, ntr = 0;
  double tdb = oracle_td(D, dtype, n, ld, med, k, NULL);
  if (k >= n) { /* every point is a medoid: nothing to swap */
    iters = 1;
    conv = 1;
  } else if (k == 1) {
    while (iters < max_iter) {
      or_key b;
      one_medoid_eval(&m, med, &b);
      iters++;
      if (!(b.delta < -tol)) {
        conv = 1;
        break;
      }
      apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, b.delta, 0, b.cand);
      med[0] = (int32_t)b.cand;
      swaps++;
      tdb += b.delta;
    }
  } else if (variant <= 2) {
    double *cd = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *cs = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    while (iters < max_iter) {
      or_key b;
      eval_all(&m, med, k, variant, cd, cs, &b);
      iters++;
      if (!(b.delta < -tol)) {
        conv = 1;
        break;
      }
      apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, b.delta, b.slot, b.cand);
      med[b.slot] = (int32_t)b.cand;
      swaps++;
      tdb += b.delta;
    }
    free(cd);
    free(cs);
  } else if (variant == 3) {
    /* FastPAM2, read as: keep the best (Delta_i*, c_i*) per slot over all
     * candidates (lowest c on ties); apply the global best (the FastPAM1
     * swap); then visit the other slots in ascending (Delta_i*, i) with
     * Delta_i* < 0, skip a slot whose c_i* is already a medoid, recompute
     * the exact Delta of that swap against the current medoids and apply it
     * iff Delta < -fp2_tol * |Delta*|.  Stop when Delta* >= -tol. */
    double *bd = (double *)malloc(sizeof(double) * (size_t)k);
    int64_t *bc = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    double *acc = (double *)malloc(sizeof(double) * (size_t)k);
    int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    double *ds = (double *)malloc(sizeof(double) * (size_t)n);
    double *rl = (double *)malloc(sizeof(double) * (size_t)k);
    char *is_med = (char *)calloc((size_t)n, 1);
    int *order = (int *)malloc(sizeof(int) * (size_t)k);
    while (iters < max_iter) {
      memset(is_med, 0, (size_t)n);
      for (int j = 0; j < k; j++) is_med[med[j]] = 1;
      oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
      oracle_removal_loss(n, k, near, dn, ds, rl);
      for (int i = 0; i < k; i++) {
        bd[i] = OR_INF;
        bc[i] = -1;
      }
      for (int64_t c = 0; c < n; c++) {
        if (is_med[c]) continue;
        double plus = 0.0;
        for (int i = 0; i < k; i++) acc[i] = rl[i];
        for (int64_t o = 0; o < n; o++) {
          double doc = od(&m, o, c);
          if (doc < dn[o]) {
            plus += doc - dn[o];
            acc[near[o]] += dn[o] - ds[o];
          } else if (doc < ds[o]) {
            acc[near[o]] += doc - ds[o];
          }
        }
        for (int i = 0; i < k; i++)
          if (acc[i] + plus < bd[i]) {
            bd[i] = acc[i] + plus;
            bc[i] = c;
          }
      }
      int bi = 0;
      for (int i = 1; i < k; i++)
        if (bd[i] < bd[bi]) bi = i;
      iters++;
      if (!(bd[bi] < -tol)) {
        conv = 1;
        break;
      }
      double dstar = bd[bi];
      apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, dstar, bi, bc[bi]);
      med[bi] = (int32_t)bc[bi];
      is_med[bc[bi]] = 1;
      swaps++;
      tdb += dstar;
      /* additional swaps, one per remaining slot */
      int no = 0;
      for (int i = 0; i < k; i++)
        if (i != bi && bd[i] < 0.0) order[no++] = i;
      for (int a = 1; a < no; a++) { /* insertion sort by (bd, i) */
        int v = order[a], b = a - 1;
        while (b >= 0 && (bd[order[b]] > bd[v] ||
                          (bd[order[b]] == bd[v] && order[b] > v))) {
          order[b + 1] = order[b];
          b--;
        }
        order[b + 1] = v;
      }
      for (int a = 0; a < no; a++) {
        int i = order[a];
        if (is_med[bc[i]]) continue;
        double d = oracle_swap_delta(D, dtype, n, ld, med, k, i, bc[i]);
        if (d < -fp2_tol * fabs(dstar)) {
          apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, d, i, bc[i]);
          is_med[med[i]] = 0;
          med[i] = (int32_t)bc[i];
          is_med[bc[i]] = 1;
          swaps++;
          tdb += d;
        }
      }
    }
    free(bd);
    free(bc);
    free(acc);
    free(near);
    free(dn);
    free(ds);
    free(rl);
    free(is_med);
    free(order);
  } else {
    /* FasterPAM, Alg. 4, read as: scan point indices p = 0, 1, 2, ...
     * cyclically, skipping current medoids; evaluate each candidate with
     * Eq. (7) against the current state and swap it with its best slot as
     * soon as that Delta < 0 (then refresh the cache and the removal loss);
     * stop when the scan returns to the index of the last swap, or after the
     * first full pass if no swap ever happened. */
    double *acc = (double *)malloc(sizeof(double) * (size_t)k);
    int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    double *ds = (double *)malloc(sizeof(double) * (size_t)n);
    double *rl = (double *)malloc(sizeof(double) * (size_t)k);
    char *is_med = (char *)calloc((size_t)n, 1);
    for (int j = 0; j < k; j++) is_med[med[j]] = 1;
    oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
    oracle_removal_loss(n, k, near, dn, ds, rl);
    int64_t last = -1; /* absolute scan position of the last swap */
    int64_t pos = 0;
    int64_t limit = (int64_t)max_iter * n;
    while (1) {
      if ((last < 0 && pos >= n) || (last >= 0 && pos >= last + n)) {
        conv = 1;
        break;
      }
      if (pos >= limit) break;
      int64_t c = pos % n;
      pos++;
      if (is_med[c]) continue;
      int slot;
      double d = fastpam1_candidate(&m, k, near, dn, ds, rl, c, acc, &slot);
      if (d < -tol) {
        apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, d, slot, c);
        is_med[med[slot]] = 0;
        med[slot] = (int32_t)c;
        is_med[c] = 1;
        swaps++;
        tdb += d;
        last = pos - 1;
        oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
        oracle_removal_loss(n, k, near, dn, ds, rl);
      }
    }
    visited = pos;
    iters = (pos + n - 1) / n;
    free(acc);
    free(near);
    free(dn);
    free(ds);
    free(rl);
    free(is_med);
  }
  stats[0] = iters;
  stats[1] = swaps;
  stats[2] = conv;
  stats[3] = visited;
  td[0] = tdb;
  td[1] = oracle_td(D, dtype, n, ld, med, k, NULL);
  return 0;
}

/* ------------------------------------------------------------------------
 * Distance-weighted initialisation (Sec. 2.3 and 3.3: the k-means++ seeding
 * with distances instead of squared distances): the first medoid is drawn
 * uniformly, every further one with probability proportional to its
 * distance to the nearest medoid drawn so far.  The uniform numbers are
 * given: u[0..k), each in [0, 1).  Draw 0 picks floor(u_0 n).  Draw t >= 1
 * uses the weights w_o = floor(d_n(o) 2^f) -- exact 64-bit fixed point with
 * f = 60 - ceil(log2(n+1)) - e(M) as for the SWAP sums (M the largest
 * entry; integer data: w_o = d_n(o)) -- their total W, the threshold
 * T = floor(u_t W) evaluated in FP64 (clamped to W - 1), and picks the
 * lowest o whose running sum of weights exceeds T.  A drawn medoid has
 * d_n = 0, so no point is drawn twice; if W = 0 the lowest-index point
 * not yet drawn is taken.  Returns 0, or -1 on invalid input.
 * ---------------------------------------------------------------------- */
static int64_t fx_weight(const or_mat *m, double x, int f) {
  if (m->dtype == 0) return (int64_t)x;
  return (int64_t)floor(ldexp(x, f)); /* x * 2^f is exact in FP64 */
}

int oracle_fixed_shift(const void *D, int dtype, int64_t n, int64_t ld) {
  if (dtype == 0) return 0;
  const float *F = (const float *)D;
  float mx = 0.0f;
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++)
      if (F[i * ld + j] > mx) mx = F[i * ld + j];
  int em = 0;
  if (mx > 0.0f) (void)frexpf(mx, &em); /* mx < 2^em */
  int bn = 0;
  while ((1ll << bn) <= (long long)n) bn++; /* n < 2^bn */
  return 60 - bn - em;
}

int oracle_init_weighted(const void *D, int dtype, int64_t n, int64_t ld, int k,
                         const double *u, int32_t *med) {
  if (k < 1 || k > n || n < 1) return -1;
  or_mat m = mk(D, dtype, n, ld);
  const int f = oracle_fixed_shift(D, dtype, n, ld);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  char *drawn = (char *)calloc((size_t)n, 1);
  int64_t c = (int64_t)floor(u[0] * (double)n);
  if (c > n - 1) c = n - 1;
  if (c < 0) c = 0;
  med[0] = (int32_t)c;
  drawn[c] = 1;
  for (int64_t o = 0; o < n; o++) dn[o] = od(&m, o, c);
  for (int t = 1; t < k; t++) {
    int64_t W = 0;
    for (int64_t o = 0; o < n; o++) W += fx_weight(&m, dn[o], f);
    int64_t pick = -1;
    if (W > 0) {
      int64_t T = (int64_t)floor(u[t] * (double)W);
      if (T > W - 1) T = W - 1;
      if (T < 0) T = 0;
      int64_t run = 0;
      for (int64_t o = 0; o < n; o++) {
        run += fx_weight(&m, dn[o], f);
        if (run > T) {
          pick = o;
          break;
        }
      }
    } else {
      for (int64_t o = 0; o < n; o++)
        if (!drawn[o]) {
          pick = o;
          break;
        }
    }
    med[t] = (int32_t)pick;
    drawn[pick] = 1;
    for (int64_t o = 0; o < n; o++) {
      const double v = od(&m, o, pick);
      if (v < dn[o]) dn[o] = v;
    }
  }
  free(dn);
  free(drawn);
  return 0;
}

/* ------------------------------------------------------------------------
 * LAB, Linear Approximative BUILD (Sec. 3.3): BUILD restricted to a fresh
 * random subsample before each medoid is chosen.  Step t (t = 0..k-1) takes
 * a subsample S_t of s points from the n - t points that are not medoids
 * yet; the candidate c in S_t with the least
 *     gain(c) = sum_{o in S_t} min(d(o,c) - d_n(o), 0)
 * (the change of the subsample's TD when c is added; d_n(o) = distance to
 * the nearest medoid chosen so far; o = c included, as in BUILD) becomes
 * the next medoid.  Step 0 has no medoid yet: gain(c) = sum_{o in S_t}
 * d(o,c), the subsample's 1-medoid.  Lowest point index on equal gains.
 *
 * The subsamples are given as ranks: rank[t*s + j] in [0, n - t), distinct
 * within a step, names the rank-th non-medoid in ascending point index at
 * step t; a negative rank is an unused entry (a smaller subsample), and a
 * step needs at least one used entry.  Gains are summed in the exact fixed point of the SWAP sums
 * (distances enter as floor(x 2^f); integer data unchanged), so the choice
 * does not depend on the summation order.  gains_out (may be NULL) gets
 * each step's least gain as a double (fixed point scaled back by 2^-f).
 * Returns 0, or -1 on invalid input (bad sizes, a rank out of range or
 * repeated within its step).
 * ---------------------------------------------------------------------- */
int oracle_init_lab(const void *D, int dtype, int64_t n, int64_t ld, int k,
                    int s, const int32_t *rank, int32_t *med,
                    double *gains_out) {
  if (k < 1 || k > n || n < 1 || s < 1) return -1;
  or_mat m = mk(D, dtype, n, ld);
  const int f = oracle_fixed_shift(D, dtype, n, ld);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  char *is_med = (char *)calloc((size_t)n, 1);
  int64_t *pts = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
  char *used = (char *)calloc((size_t)n, 1);
  int rc = 0;
  for (int64_t o = 0; o < n; o++) dn[o] = OR_INF;
  for (int t = 0; t < k && rc == 0; t++) {
    /* the subsample: rank r -> the r-th non-medoid in index order */
    int cnt = 0;
    for (int j = 0; j < s; j++) {
      const int64_t r = rank[(size_t)t * s + j];
      if (r < 0) continue; /* unused entry: a smaller subsample */
      if (r >= n - t) {
        rc = -1;
        break;
      }
      int64_t seen = -1, p = -1;
      for (int64_t o = 0; o < n; o++) {
        if (!is_med[o]) seen++;
        if (seen == r) {
          p = o;
          break;
        }
      }
      if (used[p]) {
        rc = -1;
        break;
      }
      used[p] = 1;
      pts[cnt++] = p;
    }
    for (int j = 0; j < cnt; j++) used[pts[j]] = 0;
    if (rc != 0) break;
    if (cnt == 0) {
      rc = -1; /* an empty subsample */
      break;
    }
    int64_t best = 0, pick = -1;
    for (int a = 0; a < cnt; a++) {
      const int64_t c = pts[a];
      int64_t g = 0;
      for (int b = 0; b < cnt; b++) {
        const int64_t o = pts[b];
        const int64_t dc = fx_weight(&m, od(&m, o, c), f);
        if (t == 0) {
          g += dc;
        } else {
          const int64_t v = dc - fx_weight(&m, dn[o], f);
          if (v < 0) g += v;
        }
      }
      if (pick < 0 || g < best || (g == best && c < pick)) {
        best = g;
        pick = c;
      }
    }
    med[t] = (int32_t)pick;
    is_med[pick] = 1;
    if (gains_out)
      gains_out[t] = (dtype == 0) ? (double)best : ldexp((double)best, -f);
    for (int64_t o = 0; o < n; o++) {
      const double v = od(&m, o, pick);
      if (v < dn[o]) dn[o] = v;
    }
  }
  free(dn);
  free(is_med);
  free(pts);
  free(used);
  return rc;
}

/* ------------------------------------------------------------------------
 * TD objective, Eq. (2), of medoids given as point indices of feature
 * vectors X (n x d float32, row-major), with the Euclidean distance computed
 * directly in FP64: TD = sum_o min_j sqrt(sum_t (x_o,t - x_m_j,t)^2).
 * labels (may be NULL) = lowest slot attaining the minimum.  For data
 * without a stored matrix (the on-the-fly form), this is the exact TD
 * against which the GPU's reported TD is compared.
 * ---------------------------------------------------------------------- */
double oracle_td_points(const float *X, int64_t n, int d, const int32_t *med,
                        int k, int32_t *labels) {
  double td = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : td)
  for (int64_t o = 0; o < n; o++) {
    double best = OR_INF;
    int lab = -1;
    for (int j = 0; j < k; j++) {
      const float *a = X + (size_t)o * d, *b = X + (size_t)med[j] * d;
      double s = 0.0;
      for (int t = 0; t < d; t++) {
        const double df = (double)a[t] - (double)b[t];
        s += df * df;
      }
      const double v = sqrt(s);
      if (v < best) {
        best = v;
        lab = j;
      }
    }
    td += best;
    if (labels) labels[o] = lab;
  }
  return td;
}

/* ------------------------------------------------------------------------
 * FastCLARANS (Sec. 3.4): CLARANS's randomized search with the FastPAM1
 * evaluation.  CLARANS draws a random (medoid, non-medoid) pair, swaps if
 * that lowers TD and stops after a fixed number of consecutive failed
 * draws; FastCLARANS draws only the non-medoid and evaluates it against all
 * k medoids at once.  The draws are given: cand[0..len) (a draw that is a
 * medoid at its turn is skipped and not counted).  Each draw c: Delta =
 * min over slots of Eq. (7) (lowest slot on ties); if Delta < -tol the swap
 * is applied at once (the new medoid takes the slot) and the failure count
 * restarts at 0, else it grows by one; the search stops when it reaches
 * maxneighbor or the draws run out.  Needs 2 <= k < n.
 * stats[0] = draws consumed (medoids included), stats[1] = swaps,
 * stats[2] = 1 if stopped by maxneighbor, stats[3] = draws evaluated.
 * td and the trace as in oracle_swap.  Returns 0, or -1 on invalid input.
 * ---------------------------------------------------------------------- */
int oracle_clarans(const void *D, int dtype, int64_t n, int64_t ld, int k,
                   int32_t *med, const int32_t *cand, int64_t len,
                   int64_t maxneighbor, double tol, int64_t *stats, double *td,
                   int trace_cap, double *tr_d, int32_t *tr_i, int64_t *tr_c) {
  if (k < 2 || k >= n || len < 0 || maxneighbor < 1) return -1;
  or_mat m = mk(D, dtype, n, ld);
  double *acc = (double *)malloc(sizeof(double) * (size_t)k);
  int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *dn = (double *)malloc(sizeof(double) * (size_t)n);
  double *ds = (double *)malloc(sizeof(double) * (size_t)n);
  double *rl = (double *)malloc(sizeof(double) * (size_t)k);
  char *is_med = (char *)calloc((size_t)n, 1);
  for (int j = 0; j < k; j++) is_med[med[j]] = 1;
  oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
  oracle_removal_loss(n, k, near, dn, ds, rl);
  double tdb = oracle_td(D, dtype, n, ld, med, k, NULL);
  int64_t fails = 0, pos = 0, evaluated = 0, swaps = 0, ntr = 0;
  int stopped = 0;
  while (pos < len) {
    const int64_t c = cand[pos++];
    if (c < 0 || c >= n || is_med[c]) continue;
    evaluated++;
    int slot;
    const double d = fastpam1_candidate(&m, k, near, dn, ds, rl, c, acc, &slot);
    if (d < -tol) {
      apply_trace(&ntr, trace_cap, tr_d, tr_i, tr_c, d, slot, c);
      is_med[med[slot]] = 0;
      med[slot] = (int32_t)c;
      is_med[c] = 1;
      swaps++;
      tdb += d;
      fails = 0;
      oracle_cache(D, dtype, n, ld, med, k, near, NULL, dn, ds);
      oracle_removal_loss(n, k, near, dn, ds, rl);
    } else if (++fails >= maxneighbor) {
      stopped = 1;
      break;
    }
  }
  stats[0] = pos;
  stats[1] = swaps;
  stats[2] = stopped;
  stats[3] = evaluated;
  td[0] = tdb;
  td[1] = oracle_td(D, dtype, n, ld, med, k, NULL);
  free(acc);
  free(near);
  free(dn);
  free(ds);
  free(rl);
  free(is_med);
  return 0;
}

/* ------------------------------------------------------------------------
 * Euclidean dissimilarity matrix of m float32 points in FP64, rounded once
 * to float32: D[i*ld + j] = sqrt(sum_t (x_it - x_jt)^2) (zero diagonal,
 * symmetric by construction).  The Euclidean distance written out: FP64
 * differences, their squares added one coordinate after the other in plain
 * FP64 (the oracle is built with -ffp-contract=off, so no multiply-add is
 * fused), FP64 square root, one rounding to float32.  Used for CLARA samples
 * and batch instances.
 * ---------------------------------------------------------------------- */
void oracle_euclid_f32(const float *X, int64_t m, int d, const int64_t *idx,
                       int64_t ld, float *D) {
  for (int64_t i = 0; i < m; i++) {
    const float *xi = X + (idx ? idx[i] : i) * (int64_t)d;
    for (int64_t j = 0; j < m; j++) {
      const float *xj = X + (idx ? idx[j] : j) * (int64_t)d;
      double s = 0.0;
      for (int t = 0; t < d; t++) {
        double df = (double)xi[t] - (double)xj[t];
        s += df * df;
      }
      D[i * ld + j] = (float)sqrt(s);
    }
    for (int64_t j = m; j < ld; j++) D[i * ld + j] = 0.0f;
  }
}

/* ------------------------------------------------------------------------
 * CLARA (Sec. 2.1 "Variants and Extensions of PAM", Sec. 3.4 FastCLARA):
 * for each of `samples` subsamples of s points (indices given, drawn by the
 * caller), run PAM -- BUILD then FastPAM1 -- on the subsample's matrix,
 * assign every point of the full data set to its nearest medoid, and keep
 * the medoids with the least TD on the full data (lowest sample index on
 * ties).  Distances are Euclidean in FP64 from float32 coordinates.
 * Outputs: medoids (global indices, k), labels (n, may be NULL), the TD of
 * every sample (samples) and the index of the best sample.
 * ---------------------------------------------------------------------- */
int oracle_clara(const float *X, int64_t n, int d, int k, int samples, int s,
                 const int32_t *sample_idx, int32_t *medoids, int32_t *labels,
                 double *sample_td, int32_t *best_sample) {
  int64_t ld = (s + 3) / 4 * 4;
  float *D = (float *)malloc(sizeof(float) * (size_t)s * (size_t)ld);
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
  int32_t *med = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *bestmed = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  double best_td = OR_INF;
  int best = -1;
  for (int q = 0; q < samples; q++) {
    for (int i = 0; i < s; i++) idx[i] = sample_idx[(int64_t)q * s + i];
    oracle_euclid_f32(X, s, d, idx, ld, D);
    double tdb;
    oracle_build(D, 1, s, ld, k, med, &tdb, NULL);
    int64_t stats[4];
    double tds[2];
    oracle_swap(D, 1, s, ld, k, med, 2, 100 * k + 100, 0.0, 0.0, stats, tds, 0,
                NULL, NULL, NULL);
    /* full-data TD of this sample's medoids (global indices) */
    double td = 0.0;
#pragma omp parallel for reduction(+ : td) schedule(static)
    for (int64_t o = 0; o < n; o++) {
      double b = OR_INF;
      for (int j = 0; j < k; j++) {
        const float *xm = X + (int64_t)idx[med[j]] * d;
        const float *xo = X + o * (int64_t)d;
        double sq = 0.0;
        for (int t = 0; t < d; t++) {
          double df = (double)xo[t] - (double)xm[t];
          sq += df * df;
        }
        double v = sqrt(sq);
        if (v < b) b = v;
      }
      td += b;
    }
    if (sample_td) sample_td[q] = td;
    if (td < best_td) {
      best_td = td;
      best = q;
      for (int j = 0; j < k; j++) bestmed[j] = (int32_t)idx[med[j]];
    }
  }
  for (int j = 0; j < k; j++) medoids[j] = bestmed[j];
  if (labels) {
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n; o++) {
      double b = OR_INF;
      int lab = -1;
      for (int j = 0; j < k; j++) {
        const float *xm = X + (int64_t)bestmed[j] * d;
        const float *xo = X + o * (int64_t)d;
        double sq = 0.0;
        for (int t = 0; t < d; t++) {
          double df = (double)xo[t] - (double)xm[t];
          sq += df * df;
        }
        double v = sqrt(sq);
        if (v < b) {
          b = v;
          lab = j;
        }
      }
      labels[o] = lab;
    }
  }
  if (best_sample) *best_sample = best;
  free(D);
  free(idx);
  free(med);
  free(bestmed);
  return 0;
}

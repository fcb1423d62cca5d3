/*
 * kmedoids.h -- C ABI of the GB300 (sm_103a) k-medoids library
 * (libkmedoids.so).
 *
 * The library implements the hot path of Schubert & Rousseeuw, "Fast and
 * Eager k-Medoids Clustering: O(k) Runtime Improvement of the PAM, CLARA,
 * and CLARANS Algorithms" (arXiv 2008.05171):
 *
 *   - PAM BUILD (Alg. 1), the greedy initialisation, with every candidate's
 *     gain kept exact and updated after each step from the matrix rows of
 *     the points whose nearest distance the new medoid lowered (the same
 *     choices as re-evaluating every candidate, a few matrix passes per
 *     BUILD instead of k);
 *   - the per-point cache nearest / d_n / d_s (Sec. 2) and the removal loss
 *     Delta^{-m_i} (Eq. (7));
 *   - the FastPAM1 SWAP evaluation (Alg. 3, Eq. (7)): Delta TD of every
 *     (medoid slot i, non-medoid candidate c) in O(n) per candidate;
 *   - the best swap, its application and the cache update (Alg. 3);
 *   - FastPAM2 (Sec. 3.2), the eager FasterPAM (Alg. 4) and FastCLARANS
 *     (Sec. 3.4);
 *   - the distance-weighted and LAB initialisations (Sec. 3.3);
 *   - on-the-fly distances from bf16 features on the tensor cores, many
 *     instances in one persistent launch, and CLARA (Sec. 2.1, 3.4).
 *
 * Data conventions (all entry points):
 *   D       dissimilarity matrix, n rows of ld elements, row-major, DEVICE
 *           memory owned by the caller.  d(x_o, x_c) = D[c*ld + o].  D must
 *           be symmetric with a zero diagonal and finite entries >= 0 (the
 *           paper's symmetric special case, Sec. 1.2); the library does not
 *           scan D to check this.  Columns n..ld-1 are padding and never
 *           read as distances.  The base address must be 16-byte aligned and
 *           ld a multiple of 4 (8 for KM_U16: rows are streamed with 16-byte
 *           bulk copies);
 *           otherwise the call returns KM_E_INVALID.
 *   dtype   KM_I32 (int32 distances; sums in int64, results exact),
 *           KM_U16 (uint16 distances, the compressed form; as KM_I32), or
 *           KM_F32 (float32 distances; TD sums in FP64, the SWAP Delta sums
 *           and the BUILD gains in exact 64-bit fixed point with a per-call
 *           scale 2^f, f = 60 - ceil(log2(n+1)) - (exponent of the largest
 *           entry), i.e. ~2^-(60-log2 n) resolution relative to the largest
 *           distance (the plain BUILD pass of km_options.build_full sums
 *           compensated FP32 partials in FP64); float inputs are scanned
 *           once per call and entries
 *           that are negative or not finite return KM_E_NUMERIC).
 *   medoids int32 point indices in SLOT order, DEVICE memory.  A swap puts
 *           the new medoid into the removed medoid's slot.  Labels are slots.
 *   ws      DEVICE workspace of at least kmedoids_workspace_size() bytes,
 *           256-byte aligned, owned by the caller; the library never
 *           allocates device memory for data.  What it keeps between calls
 *           is derived from arguments alone: the measured kernel geometry
 *           per shape (tune = -1) and up to 8 instantiated CUDA graphs of
 *           the FastPAM1 SWAP loop, keyed by every argument they embed.
 *   stream  a cudaStream_t (NULL = legacy default stream).  Every call
 *           enqueues its work on this stream and synchronises it before
 *           returning (the result struct is filled on the host).
 *   Ties    nearest medoid = lowest slot among equal distances; per
 *           candidate the lowest slot; the applied swap is the
 *           lexicographic minimum of (Delta, slot, candidate); BUILD takes
 *           the lowest point index among equal gains.
 *
 * Errors: every call returns a km_status and never aborts the process.
 * Arguments are validated before any work is enqueued.  A device-side wait
 * that exceeds its time limit returns KM_E_TIMEOUT.  kmedoids_last_error()
 * returns a thread-local message describing the last failure.
 */
#ifndef KMEDOIDS_H_
#define KMEDOIDS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KM_OK = 0,
  KM_E_INVALID = 1,       /* bad argument (sizes, pointers, alignment) */
  KM_E_WORKSPACE = 2,     /* workspace smaller than required */
  KM_E_CUDA = 3,          /* a CUDA runtime call failed */
  KM_E_NOT_CONVERGED = 4, /* max_iter reached; results are the best so far */
  KM_E_TIMEOUT = 5,       /* a device-side wait gave up */
  KM_E_NUMERIC = 6,       /* non-finite value met where a distance was due */
  KM_E_UNSUPPORTED = 7,   /* valid but outside the library's limits */
  KM_E_BOUNDS = 8         /* bounds-checking build only: a kernel met an
                             index out of range and skipped the access */
} km_status;

/* KM_U16: the compressed integer form -- unsigned 16-bit distances (0 ..
 * 65535; integer dissimilarities in that range lose nothing), half the
 * bytes of KM_I32 per matrix pass.  Widened to int32 in the kernels, sums
 * in int64, results exact as for KM_I32; ld must be a multiple of 8, and
 * the cache arrays kmedoids_cache returns (dn, ds) are int32.  Matrix form
 * only. */
typedef enum { KM_I32 = 0, KM_F32 = 1, KM_U16 = 2 } km_dtype;

typedef enum {
  KM_FASTPAM1 = 0, /* best swap per iteration (Alg. 3); same swaps as PAM */
  KM_FASTPAM2 = 1, /* best swap per slot, up to k swaps per iteration */
  KM_FASTERPAM = 2, /* eager: first improving candidate in scan order (Alg. 4) */
  KM_FASTCLARANS = 3 /* randomized search (Sec. 3.4): the caller's candidate
                        draws (opts->draws) in order, each evaluated against
                        all k medoids with Eq. (7) and swapped at once if it
                        improves; stops after opts->maxneighbor consecutive
                        failed draws.  Needs 2 <= k < n. */
} km_variant;

/* Options.  Zero-initialise and call km_default_options() first. */
typedef struct km_options {
  int32_t variant;        /* km_variant */
  int32_t max_iter;       /* evaluation passes (FasterPAM: full scans);
                             <= 0 means 100*k + 100 */
  double tol;             /* a swap is applied iff Delta < -tol (default 0) */
  double fastpam2_tol;    /* FastPAM2 applies an additional swap iff its
                             recomputed Delta < -fastpam2_tol * |Delta*| */
  int32_t rows_per_tile;  /* candidate rows per CTA tile; 0 = automatic.
                             FasterPAM / FastCLARANS: scan positions per
                             CTA in the longest window (0 = 8); a window
                             spans one position per CTA right after a swap
                             and doubles, up to this, while none is found.
                             They run as one persistent cooperative launch
                             (one CTA of 512 threads per SM) that
                             evaluates a window, takes the first improving
                             position and applies it without returning to
                             the host. */
  int32_t profile;        /* nonzero: time kernels with CUDA events */
  int32_t trace_capacity; /* entries available in the trace arrays */
  int32_t tune;           /* matrix-form kernel geometry (tile rows, ring
                             stages, CTAs per SM):
                             0 = automatic (the library's preference
                               order, measured on GB300 at n = 20000 and
                               50000);
                             -1 = measured: the first call for a given
                               (device, dtype, BUILD/SWAP, variant, n, k)
                               times one pass of every table entry that
                               fits on the caller's matrix and keeps the
                               fastest for the rest of the process (costs
                               three passes per entry once; results do not
                               depend on the geometry);
                             1..16 = a fixed table entry (for FasterPAM
                               and FastCLARANS: run the windowed streaming
                               kernel of that geometry, one launch per
                               window, instead of the persistent eager
                               kernel);
                             KM_E_UNSUPPORTED if it does not fit */
  /* HOST arrays (may be NULL) receiving every applied swap in order. */
  double *trace_delta;
  int32_t *trace_slot;
  int32_t *trace_cand;
  int64_t *trace_time_ns; /* device %globaltimer when the swap was applied */
  double *build_gains;    /* HOST, k entries: BUILD step gains (step 0 = the
                             first medoid's distance sum) */
  /* KM_FASTCLARANS only: */
  const int32_t *draws;   /* DEVICE, draws_len point indices (the random
                             non-medoid picks; a draw that is a medoid at
                             its turn, or out of range, is skipped) */
  int64_t draws_len;
  int64_t maxneighbor;    /* consecutive failed draws that end the search
                             (the paper samples 2.5 % of n - k) */
  int32_t check_input;    /* nonzero (kmedoids_build / _swap / _run): one
                             extra pass over D before any other work checks
                             the assumptions of the method -- zero
                             diagonal and bitwise symmetry (else
                             KM_E_INVALID) and, for KM_F32, entries finite
                             and >= 0 (else KM_E_NUMERIC); 32 x 32 tiles of
                             the upper triangle against their mirrors */
  int32_t build_full;     /* BUILD (kmedoids_build / _run):
                             0 (default) = incremental: the gains of all
                               candidates are kept in exact 64-bit fixed
                               point and, after each step, updated from the
                               matrix rows of the points whose nearest
                               distance the new medoid lowered only (a few
                               passes over D in total on clustered data
                               instead of k); for KM_F32 one extra pass
                               first finds the fixed-point scale (and
                               rejects negative, infinite or NaN entries
                               with KM_E_NUMERIC);
                             nonzero = every step streams all candidate
                               rows (the plain pass of Alg. 1, FP32 sums
                               with compensation for KM_F32).
                             Both choose the same medoids up to FP32
                             rounding of the plain pass's sums (identical
                             for integer data). */
  int64_t wait_limit_ns;  /* limit of every bounded device wait of the call
                             (pipeline stages, consumer barriers, the grid
                             barrier of the eager kernel), in nanoseconds;
                             0 = 4 s.  A wait that runs out makes the call
                             return KM_E_TIMEOUT (the kernels stop, let
                             their own copies land and release tensor
                             memory; the workspace is then undefined, the
                             matrix untouched).  Negative: KM_E_INVALID.
                             A limit far below a kernel's normal wait times
                             turns ordinary calls into timeouts. */
  int32_t swap_full;      /* SWAP of the on-the-fly form (kmedoids_run_features
                             / _swap_features, k >= 2):
                             0 (default) = incremental: every candidate's
                               per-slot sums of Eq. (7) are kept in exact
                               64-bit fixed point in the workspace; the
                               first pass sums every point, each later pass
                               only the points whose nearest / second
                               distances the last swap changed (their old
                               terms out, their new terms in), so the
                               same Delta of every swap is found at a
                               fraction of the work; the workspace holds
                               n x k_pad 64-bit sums for it;
                             nonzero = every pass sums every point (the
                               plain FastPAM1 pass).
                             Both take the same swaps (the sums are exact
                             integer functions of the same pair
                             distances).  Ignored by the matrix forms. */
  int32_t gram_full;      /* dense passes of the on-the-fly form (its first
                             BUILD step, and the swap of k = 1), which sum
                             every pair's distance for every candidate:
                             0 (default) = each 128 x 128 Gram tile pair is
                               computed once and used for both roles
                               (d(c, o) = d(o, c)): candidate tile t takes
                               the point blocks b >= t, adds each distance
                               to its row's candidate and, off the
                               diagonal, to its column's point as a
                               candidate (half the tensor-core work);
                             nonzero = every tile in both orientations.
                             The two differ only by FP32 rounding of a
                             pair's distance from the other orientation's
                             Gram entry.  Ignored by the matrix forms. */
} km_options;

/* Results, filled on the HOST before the call returns. */
typedef struct km_result {
  double td;            /* final TD = sum of d_n, recomputed on the device
                           (FP64 for KM_F32, exact for KM_I32) */
  int64_t td_i64;       /* final TD as int64 (KM_I32 only) */
  double td_bookkept;   /* initial TD + sum of the applied Delta values */
  double td_initial;    /* TD of the starting medoids (after BUILD) */
  int32_t iterations;   /* evaluation passes (FasterPAM: scans started;
                           FastCLARANS: draws evaluated) */
  int32_t swaps;        /* swaps applied */
  int32_t status;       /* km_status of the call */
  int32_t build_steps;  /* medoids chosen by BUILD */
  int64_t visited;      /* FasterPAM: scan positions visited; FastCLARANS:
                           draws consumed (KM_E_NOT_CONVERGED if the draws
                           ran out before maxneighbor consecutive failures) */
  /* profile != 0 only (milliseconds of device time, CUDA events): */
  double build_ms;      /* whole BUILD */
  double swap_ms;       /* whole SWAP phase (cache init + iterations) */
  double eval_ms;       /* sum over the SWAP evaluation kernel launches */
  int32_t eval_launches;
  int32_t build_launches; /* BUILD evaluation kernel launches */
  double build_eval_ms;   /* sum over the BUILD evaluation kernel launches */
  int64_t kernel_launches; /* kernels this call launched (all phases) */
  int32_t best_sample;     /* kmedoids_clara: index of the winning sample */
  int16_t swap_geometry;   /* geometry table entries (1..16) the SWAP and */
  int16_t build_geometry;  /* BUILD passes ran with; 0 = not run, (SWAP)
                              the eager kernel of FasterPAM / FastCLARANS,
                              or (BUILD) the incremental BUILD, whose launch
                              shape is fixed (opts->tune then applies to
                              the SWAP passes only) */
  int64_t evaluated;       /* FasterPAM / FastCLARANS: candidates evaluated
                              by the sequential scan (non-medoid positions
                              up to each applied swap, and every position
                              of the passes without one); each costs one
                              pass over the n points */
  int64_t build_rows;      /* rows of D (n elements each) the BUILD
                              evaluation kernels streamed */
  double eval_ms_median;   /* profile != 0: median over the SWAP evaluation
                              launches of their device time */
  double eval_ms_first;    /* profile != 0: device time of the first SWAP
                              evaluation launch (the on-the-fly form's
                              incremental SWAP: the pass over every point;
                              the later ones move the changed points only) */
} km_result;

/* Parameters of a matrix-form geometry table entry (1..16, as reported in
 * km_result.swap_geometry / build_geometry and accepted by opts->tune):
 * candidate rows per tile, shared-memory ring stages, CTAs per SM.  A pass
 * launches min(SMs x ctas_per_sm, ceil(n / rows), 1024) CTAs.  Returns 0,
 * or 1 for an unknown entry (outputs untouched; NULL outputs skipped). */
int kmedoids_geometry_info(int32_t geometry, int32_t *rows, int32_t *stages,
                           int32_t *ctas_per_sm);

/* Fill *o with the defaults (FastPAM1, tol 0, automatic tiles). */
void km_default_options(km_options *o);

/* Bytes of device workspace the calls below need for (n, k, dtype, options)
 * (the trace capacity and FastPAM2's per-slot partials depend on them).
 * Returns 0 for invalid sizes. */
size_t kmedoids_workspace_size(int64_t n, int32_t k, int32_t dtype,
                               const km_options *opts);

/* PAM BUILD (Alg. 1): k greedy steps.  Step 0 takes the point with the
 * smallest distance sum (the 1-medoid, Eq. (3)); each further step adds the
 * non-medoid c minimising sum_o min(d(o,c) - d_n(o), 0), the exact TD change
 * of adding c (the point c itself included; lowest index on ties).  By
 * default the gains of all candidates are kept and updated after each step
 * from the rows of the points whose d_n the new medoid lowered (see
 * km_options.build_full).  Writes k medoids (slot order = order chosen) to
 * medoids_out (DEVICE).  res->td = TD of the result; res->build_rows = rows
 * of D the BUILD streamed. */
km_status kmedoids_build(const void *D, int32_t dtype, int64_t n, int64_t ld,
                         int32_t k, int32_t *medoids_out,
                         const km_options *opts, km_result *res, void *ws,
                         size_t ws_bytes, void *stream);

/* SWAP (Alg. 3 / Sec. 3.2 / Alg. 4, by opts->variant) from the k medoids in
 * medoids_inout (DEVICE, updated in place) until no swap has Delta < -tol
 * or max_iter passes were made (KM_E_NOT_CONVERGED).  labels_out (DEVICE,
 * n entries, may be NULL) receives each point's nearest slot at exit.
 * k = 1 swaps directly to the 1-medoid (Eq. (3)); k = n does nothing. */
km_status kmedoids_swap(const void *D, int32_t dtype, int64_t n, int64_t ld,
                        int32_t k, int32_t *medoids_inout, int32_t *labels_out,
                        const km_options *opts, km_result *res, void *ws,
                        size_t ws_bytes, void *stream);

/* BUILD followed by SWAP; medoids_out (DEVICE, k entries). */
km_status kmedoids_run(const void *D, int32_t dtype, int64_t n, int64_t ld,
                       int32_t k, int32_t *medoids_out, int32_t *labels_out,
                       const km_options *opts, km_result *res, void *ws,
                       size_t ws_bytes, void *stream);

/* One FastPAM1 evaluation pass (Alg. 3, Eq. (7)) for the medoids given
 * (DEVICE, k entries, unchanged): for every point c, cand_delta[c] (DEVICE
 * double, n entries, may be NULL) = min_i Delta(i, c) and cand_slot[c]
 * (DEVICE int32, may be NULL) = the lowest slot attaining it; medoid rows
 * get +inf and -1.  best (HOST) receives the lexicographic minimum
 * (Delta, slot, candidate) over all non-medoids; with k = n it is
 * (+inf, -1, -1).  Requires 2 <= k <= n. */
km_status kmedoids_eval_swaps(const void *D, int32_t dtype, int64_t n,
                              int64_t ld, int32_t k, const int32_t *medoids,
                              double *cand_delta, int32_t *cand_slot,
                              double *best_delta, int32_t *best_slot,
                              int32_t *best_cand, void *ws, size_t ws_bytes,
                              void *stream);

/* The per-point cache (Sec. 2) for the medoids given: near/sec (DEVICE
 * int32, n entries) = nearest and second-nearest slot, dn/ds (DEVICE, n
 * entries, D's dtype; int32 for KM_U16) = their distances; removal
 * (DEVICE double, k entries, may be NULL) = Delta^{-m_i} of Eq. (7).  For
 * k = 1, sec = -1 and ds = the dtype's largest value.  Requires
 * 1 <= k <= n. */
km_status kmedoids_cache(const void *D, int32_t dtype, int64_t n, int64_t ld,
                         int32_t k, const int32_t *medoids, int32_t *near,
                         int32_t *sec, void *dn, void *ds, double *removal,
                         void *ws, size_t ws_bytes, void *stream);

/* Distance-weighted initialisation (Sec. 3.3; the k-means++ seeding of
 * Sec. 2.3 with distances, not squared distances, as weights): k starting
 * medoids for SWAP, typically FasterPAM (Sec. 4.3, Sec. 6), at O(nk) cost
 * instead of BUILD's O(n^2 k).
 *   u            DEVICE, k doubles in [0, 1): the caller's uniform random
 *                numbers (any generator); draw t consumes u[t].
 *   medoids_out  DEVICE, k int32: the draws in order (distinct points).
 * Draw 0 is point floor(u[0] n).  Draw t >= 1 weighs every point o by its
 * distance to the nearest medoid drawn so far, in the exact fixed point of
 * the SWAP sums (w_o = floor(d 2^f) for KM_F32, d itself for KM_I32), and
 * takes the lowest o whose running weight sum exceeds floor(u[t] W) (W the
 * total weight, product in FP64); drawn points weigh 0 and are never drawn
 * again; if W = 0 the lowest undrawn point is taken.  ws: as
 * kmedoids_workspace_size(n, k, dtype, NULL).  KM_E_INVALID for a NULL
 * pointer, a u[t] outside [0, 1) or the common size checks; KM_E_NUMERIC
 * for negative or non-finite float entries.  Synchronises the stream. */
km_status kmedoids_init_weighted(const void *D, int32_t dtype, int64_t n,
                                 int64_t ld, int32_t k, const double *u,
                                 int32_t *medoids_out, void *ws,
                                 size_t ws_bytes, void *stream);

/* LAB, Linear Approximative BUILD (Sec. 3.3): before each of the k choices
 * a fresh subsample of the points that are not medoids yet is drawn, and
 * BUILD's gain (Alg. 1) is evaluated over that subsample only; the paper
 * uses subsamples of 10 + ceil(sqrt(n)) points.
 *   s            entries per subsample (1 <= s <= 4096; k <= 8192).
 *   ranks        DEVICE, k x s int32, row t = the subsample of step t as
 *                ranks among the n - t current non-medoids in ascending
 *                point index (rank r = the (r+1)-th smallest non-medoid),
 *                distinct within a row; a negative entry is unused (a
 *                smaller subsample), every row needs one used entry.
 *   medoids_out  DEVICE, k int32: the choices in order.
 *   gains_host   HOST, k doubles (may be NULL): each step's least gain,
 *                sum_{o in S} min(d(o,c) - d_n(o), 0), and at step 0 the
 *                chosen point's distance sum over its subsample.
 * Each subsample point c is scored with that gain (its own term included,
 * as in BUILD) in the exact fixed point of the SWAP sums; the least gain
 * wins, lowest point index on ties.  ws: as kmedoids_workspace_size(n, k,
 * dtype, NULL).  KM_E_INVALID for a rank outside [0, n - t), a repeated
 * rank, an empty row, a NULL pointer or the common size checks;
 * KM_E_UNSUPPORTED beyond the s and k limits.  Synchronises the stream. */
km_status kmedoids_init_lab(const void *D, int32_t dtype, int64_t n,
                            int64_t ld, int32_t k, int32_t s,
                            const int32_t *ranks, int32_t *medoids_out,
                            double *gains_host, void *ws, size_t ws_bytes,
                            void *stream);

/* Tensor-core Gram product G = X X^T of bf16 feature vectors (tcgen05 MMA,
 * FP32 accumulation), the dot products behind the on-the-fly distances
 * d(o,c)^2 = |x_o|^2 + |x_c|^2 - 2 x_o.x_c (Sec. 4.8 notes that recomputing
 * distances instead of storing the matrix is the memory-saving option).
 * X: n rows of ldx bf16 elements (DEVICE, 16-byte aligned, ldx % 8 == 0),
 * d = 16, 32, ..., 256 features.  G: n x n FP32 (DEVICE, row stride ldg).
 * ws (DEVICE, 256-byte aligned) >= 256 + roundup(n,128) * d * 2 bytes holds
 * the operands rearranged for the tensor cores.  n <= 2^20. */
km_status kmedoids_gram_bf16(const void *X, int64_t n, int32_t d, int64_t ldx,
                             float *G, int64_t ldg, void *ws, size_t ws_bytes,
                             void *stream);

/* ---- On-the-fly distance form (no n x n matrix).  Points are n rows of d
 * bf16 features (DEVICE, row stride ldx elements, ldx % 8 == 0, 16-byte
 * aligned, d a multiple of 16 up to 240); d(o,c) is the Euclidean distance.
 * Every BUILD step and SWAP pass recomputes the distances it needs from a
 * tensor-core Gram product (tcgen05, BF16 inputs, FP32 accumulation):
 * d^2 = |x_o|^2 + |x_c|^2 - 2 x_o.x_c, the operands carrying 16 more
 * columns for |x_c|^2 / 2 and a per-point threshold (exact sums of three
 * bf16 pieces).  By default (build_full = swap_full = 0) both phases are
 * incremental: BUILD's step 0 and SWAP's first pass take every point, and
 * each later step or pass only the points the last commit or swap changed,
 * the candidates' gains and Eq. (7) sums being kept in the workspace; the
 * threshold columns are then zero, so a pair's Gram entry is the same in
 * every pass, and the kept sums equal a full recomputation's.  With
 * build_full / swap_full every step or pass takes every point and the
 * threshold test is folded into the product (the sign of one MMA output
 * decides a pair).  BUILD's step 0 (and the swap of k = 1), where every
 * pair counts for both of its points, computes each Gram tile pair once
 * and sums its distances along rows and columns (unless opts->gram_full).
 * The per-point cache (nearest, d_n,
 * d_s) and the TD are computed exactly from FP32 differences sum (x - y)^2,
 * so the Gram form's rounding (relative error ~1e-5 on d^2 for well
 * separated points) only affects which candidates see a hit and the Delta
 * values, not the cache or the reported TD.  BUILD gains, removal losses
 * and every Delta are sums of exact 64-bit fixed-point terms round(x 2^q)
 * (q per call: the diameter of the data's bounding box is below 2^25
 * units), so they do not depend on the order of the GPU's additions.
 * FastPAM1 only; k <= 224.
 * Workspace (DEVICE, 256-byte aligned): kmedoids_features_workspace_size()
 * bytes, which includes the features rearranged for the tensor cores, the
 * totals of the symmetric step 0 (8 n bytes) and, unless opts->swap_full,
 * the kept SWAP sums (8 n k_pad bytes). */
size_t kmedoids_features_workspace_size(int64_t n, int32_t d, int32_t k,
                                        const km_options *opts);

/* BUILD (Alg. 1) then FastPAM1 SWAP (Alg. 3) on the features; medoids_out
 * (DEVICE, k), labels_out (DEVICE, n, may be NULL).  res->td is the exact
 * FP32-difference TD accumulated in FP64. */
km_status kmedoids_run_features(const void *X_bf16, int64_t n, int32_t d,
                                int64_t ldx, int32_t k, int32_t *medoids_out,
                                int32_t *labels_out, const km_options *opts,
                                km_result *res, void *ws, size_t ws_bytes,
                                void *stream);

/* BUILD (Alg. 1) alone on the features: medoids_out (DEVICE, k) in the
 * order chosen; opts->build_gains receives each step's gain; labels_out
 * (DEVICE, n, may be NULL) the nearest slot of every point. */
km_status kmedoids_build_features(const void *X_bf16, int64_t n, int32_t d,
                                  int64_t ldx, int32_t k, int32_t *medoids_out,
                                  int32_t *labels_out, const km_options *opts,
                                  km_result *res, void *ws, size_t ws_bytes,
                                  void *stream);

/* FastPAM1 SWAP on the features from the medoids in medoids_inout. */
km_status kmedoids_swap_features(const void *X_bf16, int64_t n, int32_t d,
                                 int64_t ldx, int32_t k,
                                 int32_t *medoids_inout, int32_t *labels_out,
                                 const km_options *opts, km_result *res,
                                 void *ws, size_t ws_bytes, void *stream);

/* ---- Batched form: many independent PAM instances in one persistent launch.
 * Instance i's matrix lives in a float32 arena (DEVICE) at element offset
 * inst[i].offset: n rows of ld elements (ld % 4 == 0, offset % 4 == 0,
 * arena 16-byte aligned), symmetric with a zero diagonal.  Each instance
 * runs BUILD (Alg. 1) then FastPAM1 SWAP (Alg. 3) to convergence on one
 * CTA, instances taken largest first; limits n <= 4096, k <= 128.  Results
 * per instance: k medoids at medoids_out[inst[i].medoid_offset ...] and a
 * km_batch_result (exact TD of the result in FP64, passes, swaps, status). */
typedef struct km_instance {
  int64_t offset;        /* first element of the instance's matrix */
  int32_t n, ld, k;
  int32_t medoid_offset; /* where its k medoids are written */
} km_instance;

typedef struct km_batch_result {
  double td;
  int32_t iterations, swaps, status, pad;
} km_batch_result;

size_t kmedoids_batched_workspace_size(int32_t count);

/* Fill the arena with Euclidean matrices of float32 points: FP64
 * differences, squares accumulated with fused multiply-adds in coordinate
 * order, FP64 square root, one rounding to float32 (padding columns zero).
 * Instance i uses the n_i points starting at row point_offsets[i] (DEVICE
 * int64) of points (DEVICE, dim floats per point).  count <= 65535,
 * dim <= 864 (else KM_E_UNSUPPORTED).  Synchronises the stream. */
km_status kmedoids_batched_distances(const float *points, int32_t dim,
                                     const int64_t *point_offsets,
                                     const km_instance *inst, int32_t count,
                                     float *arena, void *stream);

/* inst (DEVICE, count entries, 1 <= count <= 65535), medoids_out / results
 * (DEVICE).  opts: max_iter, tol; tune 0 = geometry 1 of the persistent
 * kernel, 1 .. 5 = that geometry (see kmedoids_batched_geometry_info and
 * kmedoids_batched_autotune), anything else KM_E_INVALID;
 * variant KM_FASTPAM1 (default) or KM_FASTERPAM (Alg. 4: each CTA scans its
 * instance cyclically in windows of one candidate row per warp and applies
 * the first improving swap at once, with an incremental cache update; the
 * result's iterations then count the scans started); other variants give
 * KM_E_UNSUPPORTED.
 * Asynchronous: the call only enqueues work on the stream (a zeroing copy,
 * a kernel ordering the instances largest first, and the persistent PAM
 * kernel) and never reads device memory on the host, so it can be captured
 * in a CUDA graph.  Instances are validated on the device: one violating
 * the limits above gets status KM_E_INVALID in its result and the others
 * still run.  Host-side failures (NULL pointers, alignment, count,
 * workspace) are returned before anything is enqueued. */
km_status kmedoids_run_batched(const float *arena, const km_instance *inst,
                               int32_t count, int32_t *medoids_out,
                               km_batch_result *results,
                               const km_options *opts, void *ws,
                               size_t ws_bytes, void *stream);

/* kmedoids_run_batched without BUILD: every instance starts from the k
 * medoids the caller wrote at medoids_inout[inst[i].medoid_offset ...]
 * (DEVICE) and runs FastPAM1 (or, with opts->variant = KM_FASTERPAM,
 * FasterPAM) SWAP to convergence, the result replacing them.
 * For restarts from random starts (the paper recommends uniform random
 * initialisation with several restarts once swapping is cheap, Sec. 4.3
 * and Sec. 6): several instances may share one matrix (same offset), one
 * per starting set; the caller keeps the result with the least TD.
 * Starting medoids out of range or repeated give that instance
 * KM_E_INVALID.  Same limits, workspace and asynchrony as
 * kmedoids_run_batched. */
km_status kmedoids_swap_batched(const float *arena, const km_instance *inst,
                                int32_t count, int32_t *medoids_inout,
                                km_batch_result *results,
                                const km_options *opts, void *ws,
                                size_t ws_bytes, void *stream);

/* Geometry g (1 .. 5) of the batched form's persistent kernel: warps per
 * CTA and cp.async ring stages of 512 columns per warp.  Returns 0, or -1
 * for a g outside the table. */
int32_t kmedoids_batched_geometry_info(int32_t geometry, int32_t *warps,
                                       int32_t *stages);

/* Measured choice of the batched kernel's geometry (the tile shape of the
 * batched form: how many candidate rows a CTA streams at once and how deep
 * each warp's ring is).  Runs kmedoids_run_batched on the caller's batch
 * with every geometry of the table (one warm-up and one timed run each;
 * the outputs are overwritten with identical results, since results do not
 * depend on the geometry) and returns the fastest in *geometry_out, to be
 * passed as opts->tune to later calls (which may then be captured in a
 * CUDA graph).  ms_out (HOST, 5 entries, may be NULL) receives each
 * geometry's time (-1 if it could not launch).  The choice is cached per
 * device, variant and histogram of the instance sizes (instances counted
 * per (floor(log2 n), floor(log2 k)) bucket): with ms_out NULL a cached
 * choice is returned without measuring.  Reads the instance table back to
 * the host and synchronises the stream; arguments as kmedoids_run_batched. */
km_status kmedoids_batched_autotune(const float *arena, const km_instance *inst,
                                    int32_t count, int32_t *medoids_out,
                                    km_batch_result *results,
                                    const km_options *opts, void *ws,
                                    size_t ws_bytes, void *stream,
                                    int32_t *geometry_out, double *ms_out);

/* ---- CLARA (Sec. 2.1; FastCLARA, Sec. 3.4).  X: n points of d float32
 * features (DEVICE, row-major).  sample_idx (DEVICE, samples x
 * sample_size int32): the caller's subsamples (the paper suggests
 * sample_size = 80 + 4k).  Each sample's Euclidean matrix is built in FP64
 * and rounded to float32, solved by BUILD + FastPAM1 (batched form), and
 * every point is assigned to the sample's medoids (FP32 differences, FP64
 * TD).  The sample with the least TD wins (lowest index on ties):
 * medoids_out (DEVICE, k point indices), labels_out (DEVICE, n, may be
 * NULL), sample_td_host (HOST, samples, may be NULL); res->td = best TD,
 * res->best_sample its index.  Limits: 1 <= k <= sample_size <= min(n,
 * 4096), k <= 128, d <= 864, 16 k ceil(d/4) <= 200 KB.  Synchronises the
 * stream; a sample whose PAM run failed makes the call return its status. */
size_t kmedoids_clara_workspace_size(int32_t k, int32_t samples,
                                     int32_t sample_size);
km_status kmedoids_clara(const float *X, int64_t n, int32_t d, int32_t k,
                         int32_t samples, int32_t sample_size,
                         const int32_t *sample_idx, int32_t *medoids_out,
                         int32_t *labels_out, double *sample_td_host,
                         km_result *res, void *ws, size_t ws_bytes,
                         void *stream);

/* CLARA's outcome in device memory (kmedoids_run_batched_clara). */
typedef struct km_clara_result {
  double td;           /* full-data TD of the winning sample's medoids */
  int32_t best_sample; /* its index (lowest on ties) */
  int32_t status;      /* KM_OK, or the first failing sample's status */
} km_clara_result;

/* A batch of independent instances (as kmedoids_run_batched; count may be
 * 0) and CLARA (as kmedoids_clara) in one asynchronous enqueue: the sample
 * matrices, ONE persistent PAM launch over the batch and the samples
 * together (largest first; with opts->variant = KM_FASTERPAM the batch runs
 * FasterPAM in a launch of its own and the samples BUILD + FastPAM1), the
 * full-data assignment of every sample, the choice of the best sample and
 * the labels, all on the device.  Nothing is read back and nothing
 * synchronises, so the whole call can be captured in a CUDA graph and
 * replayed.  Outputs (DEVICE): the batch's medoids and results as
 * kmedoids_run_batched; clara_medoids_out (k point indices),
 * clara_labels_out (n, may be NULL), sample_td (samples FP64 TDs, may be
 * NULL), clara_result (one record).  opts: as kmedoids_run_batched (tune
 * picks the geometry for both); count + samples <= 65535.  Workspace
 * (DEVICE, 256-byte aligned): kmedoids_batched_clara_workspace_size(). */
size_t kmedoids_batched_clara_workspace_size(int32_t count, int32_t k,
                                             int32_t samples,
                                             int32_t sample_size);
km_status kmedoids_run_batched_clara(
    const float *arena, const km_instance *inst, int32_t count,
    int32_t *medoids_out, km_batch_result *results, const float *X, int64_t n,
    int32_t d, int32_t k, int32_t samples, int32_t sample_size,
    const int32_t *sample_idx, int32_t *clara_medoids_out,
    int32_t *clara_labels_out, double *sample_td, km_clara_result *clara_result,
    const km_options *opts, void *ws, size_t ws_bytes, void *stream);

/* kmedoids_eval_swaps without a caller-provided workspace, for callers that
 * cannot allocate device memory when they evaluate swaps (a frozen memory
 * pool, a plugin that must not use the host application's allocator, a
 * real-time loop that cannot risk a blocking allocation).  The paper has no
 * counterpart: this is a deployment interface of this library.
 * Same arguments and results as kmedoids_eval_swaps, without ws/ws_bytes.
 * Scratch: a fixed 2 MiB array in device memory that is part of the
 * library image; every GPU that loads the library holds it until the
 * process exits.  Limits: n <= 32768 and k <= 512 (larger sizes return
 * KM_E_UNSUPPORTED with a message; nothing is launched).  Allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress).  Like kmedoids_eval_swaps the call synchronises
 * the stream to return its results, so it cannot be captured in a CUDA
 * graph.  All calls share the one array: the call clears what must start
 * at zero, but calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
km_status kmedoids_eval_swaps_static(const void *D, int32_t dtype, int64_t n,
                                     int64_t ld, int32_t k,
                                     const int32_t *medoids,
                                     double *cand_delta, int32_t *cand_slot,
                                     double *best_delta, int32_t *best_slot,
                                     int32_t *best_cand, void *stream);

/* The bichromatic case (the paper's Outlook): the medoids are chosen among
 * m possible locations and the objective sums over n consumers, TD =
 * sum_c min_j d(x_c, m_j) (Eq. (2) over the consumers); with k = 1 the
 * result is the bichromatic medoid argmin_l sum_c d(x_c, x_l).
 *   D      m rows (locations) of ld elements, DEVICE, caller-owned:
 *          d(x_c, x_l) = D[l * ld + c] for consumers c < n; entries >= 0
 *          (float: finite); no symmetry or diagonal is assumed.  Same dtype,
 *          alignment and ld rules as the square form (ld >= n).
 *   k      1 <= k <= m; medoids_out[k] location indices in slot order,
 *          labels_out[n] (may be NULL) the nearest slot of every consumer.
 * kmedoids_run_bichromatic: BUILD (Alg. 1; the plain pass over every
 * non-medoid location per step) then SWAP; kmedoids_swap_bichromatic: SWAP
 * from the given locations (validated: in range, distinct).  SWAP variants
 * as km_options.variant: FastPAM1 (Alg. 3 over the consumers), FastPAM2,
 * FasterPAM and FastCLARANS (draws are location indices) in the windowed
 * streaming kernel.  check_input must be 0.  The workspace comes from
 * kmedoids_bichromatic_workspace_size; results, errors and synchronisation
 * as kmedoids_run.  The paper leaves this case unspecified beyond the
 * definition; every step is the square case's with candidates over the
 * locations and points over the consumers. */
size_t kmedoids_bichromatic_workspace_size(int64_t m, int64_t n, int32_t k,
                                           int32_t dtype,
                                           const km_options *opts);
km_status kmedoids_run_bichromatic(const void *D, int32_t dtype, int64_t m,
                                   int64_t n, int64_t ld, int32_t k,
                                   int32_t *medoids_out, int32_t *labels_out,
                                   const km_options *opts, km_result *res,
                                   void *ws, size_t ws_bytes, void *stream);
km_status kmedoids_swap_bichromatic(const void *D, int32_t dtype, int64_t m,
                                    int64_t n, int64_t ld, int32_t k,
                                    int32_t *medoids_inout, int32_t *labels_out,
                                    const km_options *opts, km_result *res,
                                    void *ws, size_t ws_bytes, void *stream);

/* The dissimilarity matrix from host memory into a device buffer (the
 * input of every entry point above; the paper's method starts from the
 * matrix, Sec. 1.2).  Copies n rows of n elements of type dtype from host
 * (row pitch host_ld elements) to D (row pitch ld elements, DEVICE memory
 * owned by the caller, n * ld elements); columns n .. ld-1 of D are set to
 * zero.  host_ld >= n and ld >= n.
 *
 * When host is page-locked memory (cudaHostAlloc, cudaMallocHost or
 * cudaHostRegister, one allocation holding every row read) the SMs read it
 * directly over the CPU-GPU link with 16-byte loads where both pitches and
 * bases allow (4- or 2-byte loads otherwise); any other host memory is
 * copied with cudaMemcpy2DAsync.  A device address returns KM_E_INVALID.
 * The call enqueues on stream and synchronises it, so host may be reused
 * on return. */
km_status kmedoids_upload_matrix(const void *host, int64_t host_ld,
                                 int32_t dtype, int64_t n, void *D,
                                 int64_t ld, void *stream);

/* kmedoids_upload_matrix for a matrix of `rows` rows of n elements (the m
 * location rows of the bichromatic form): D holds rows * ld elements. */
km_status kmedoids_upload_rows(const void *host, int64_t host_ld,
                               int32_t dtype, int64_t rows, int64_t n,
                               void *D, int64_t ld, void *stream);

/* Self-test of the bounded device waits (failure detection; the paper has
 * no counterpart).  Launches a kernel whose wait can never be satisfied,
 * built on the same wait routines the pipelined kernels use:
 *   kind 0  an mbarrier phase that nothing completes (the stage waits of
 *           the streaming and on-the-fly kernels);
 *   kind 1  a consumer barrier one of whose two warps never arrives;
 *   kind 2  the grid barrier of the eager kernel, over two CTAs of which
 *           one never arrives;
 *   kind 3  not a wait: the kernels' index check (KM_INB) applied to the
 *           index 5 and the bound 3, no memory accessed with it.  Returns
 *           KM_E_BOUNDS, with the index, the bound and the place of the
 *           check in kmedoids_last_error(), in the bounds-checking build
 *           (kmedoids_bounds_checked() = 1); KM_OK in the regular build,
 *           whose checks compile to nothing.
 * Each wait gives up after limit_ns (1 .. 10^10 ns; 0 = the default 4 s),
 * records KM_E_TIMEOUT in the device state record at the start of ws (a
 * DEVICE buffer of at least 512 bytes, 256-byte aligned, caller-owned) and
 * returns; nothing is left in flight and the CUDA context stays usable.
 * The call synchronises the stream and returns the status the device
 * recorded: KM_E_TIMEOUT when the wait ran out as designed (with the limit
 * in kmedoids_last_error()), KM_E_INVALID for a bad argument. */
km_status kmedoids_wait_selftest(int32_t kind, int64_t limit_ns, void *ws,
                                 size_t ws_bytes, void *stream);

/* 1 in the bounds-checking build of the library (libkmedoids_bounds.so,
 * compiled with -DKM_BOUNDS_CHECK), 0 in the regular build.  In the
 * bounds-checking build every kernel checks each index it loads from
 * memory (medoids, nearest / second slots, candidates, BUILD list entries,
 * initialisation picks) against the array it indexes; an index out of
 * range is recorded (KM_E_BOUNDS, with the index, its bound and the source
 * line in kmedoids_last_error()) and the access is skipped. */
int32_t kmedoids_bounds_checked(void);

/* Thread-local description of the last failure ("" if none). */
const char *kmedoids_last_error(void);

/* Library version string. */
const char *kmedoids_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KMEDOIDS_H_ */

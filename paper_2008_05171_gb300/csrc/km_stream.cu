// km_stream.cu -- the streaming kernel behind both hot loops of the method:
//
//   * SWAP evaluation (FastPAM1, Alg. 3 / Eq. (7)): for each non-medoid
//     candidate c, one pass over all points o accumulates the shared term
//     Delta^{+x_c} and the k per-slot corrections; the slot with the
//     smallest removal loss + correction wins, the shared term is added and
//     the best (Delta, slot, candidate) is reduced over the grid.
//   * BUILD evaluation (Alg. 1): for each non-medoid candidate c the gain
//     sum_o min(d(o,c) - d_n(o), 0) (step 0: the distance sum), reduced to
//     the best (gain, c).
//
// Both stream the candidate rows of the symmetric dissimilarity matrix
// (d(x_o, x_c) = D[c*ld + o]) exactly once per pass.  Each CTA owns a
// contiguous range of candidate rows.  One producer thread stages tiles of
// R rows x 1024 columns (plus the per-point cache of those columns) into a
// ring of S shared-memory stages with 1-D bulk copies (cp.async.bulk,
// completion on an mbarrier); eight consumer warps each own 4 columns per
// stage and walk the R rows.  The SWAP per-slot accumulators live in shared
// memory (FP64 for float data, int64 for integer data); the fast path of an
// element is one comparison d < d_s, which fails for most (o, c) pairs.
#define KM_SRC_ID 1  // names this file in bounds-check reports
#include <cfloat>
#include <type_traits>

#include "km_device.cuh"
#include "km_internal.h"

namespace km {

template <class T>
struct V4;
template <>
struct V4<float> {
  using type = float4;
};
template <>
struct V4<int32_t> {
  using type = int4;
};

// ------------------------------------------------------- shared layout
struct StageHdr {
  int rows[kMaxRows];    // candidate point indices of the tile
  int outidx[kMaxRows];  // output indices (row, or window offset)
  int nrows;             // 0 = end of work
  int chunk;             // column chunk j
  int first;             // j == 0
  int last;              // j == last chunk
};
static_assert(sizeof(StageHdr) <= 256, "stage header");

constexpr int kQueue = 256;  // SWAP hit descriptors per warp queue

struct Layout {
  size_t bars, flags, wkeys, rl, red, tile_rows, acc, slot_local, queues, stages;
  size_t stage_bytes, meta_bytes, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Offsets of the dynamic shared-memory regions (bytes).
__host__ __device__ inline Layout make_layout(int mode, int R, int S, int k, int fp2,
                                              int esize = 4) {
  Layout L;
  size_t o = 0;
  L.bars = o;
  o += 8 * (2 * (size_t)S + 1);  // full[S], empty[S], consumer barrier
  L.flags = o;
  o += 16;
  o = align_up(o, 16);
  L.wkeys = o;
  o += 16 * kConsWarps;
  L.rl = o;
  o += (mode == kModeSwap) ? 8 * (size_t)k : 0;
  o = align_up(o, 16);
  L.red = o;
  o += (mode == kModeBuild) ? 8 * (size_t)kConsWarps * R : 0;
  L.tile_rows = o;
  o += 4 * kMaxRows;
  o = align_up(o, 16);
  L.acc = o;
  o += (mode == kModeSwap) ? 8 * (size_t)R * (k + 1) : 0;
  L.slot_local = o;
  o += (mode == kModeSwap && fp2) ? 16 * (size_t)k : 0;
  o = align_up(o, 16);
  L.queues = o;
  o += (mode == kModeSwap) ? 2 * (size_t)kQueue * kConsWarps : 0;
  o = align_up(o, 128);
  L.stages = o;
  L.meta_bytes = (mode == kModeSwap) ? 3 * 4 * (size_t)kChunk : 4 * (size_t)kChunk;
  L.stage_bytes = 256 + L.meta_bytes + (size_t)esize * R * kChunk;
  o += L.stage_bytes * S;
  L.total = o;
  return L;
}

// --------------------------------------------------------------- kernel
// Elements of a SWAP pass that fell below d_s(o): the candidate would be
// nearest (case (i) of Alg. 3) or second nearest (case (ii)).  Terms are
// added in fixed point (Tr<T>::fx) to the candidate's row of accumulators:
// slot k holds the shared term Delta^{+x_c}, slot near(o) the correction.
//
// Hits are rare (about 1-2 % of the pairs on clustered data) but most warp
// rows hold one, so handling them where they occur would cost a whole warp
// instruction stream per hit.  Instead each lane records its hits of the
// stage in a 64-bit mask (bit 4r + j: row r, element j of its float4); at
// the end of the stage a warp prefix sum gives every hit a slot in the
// warp's queue in shared memory and all 32 lanes drain the queue together.
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class E>
__device__ __forceinline__ void swap_hit_at(int r, int col, const E* data,
                                            const unsigned char* meta, long long* acc, int k,
                                            int f, KmState* st) {
  using T = typename Val<E>::type;
  const T d = (T)data[(size_t)r * kChunk + col];
  const T dn = reinterpret_cast<const T*>(meta)[col];
  const T ds = reinterpret_cast<const T*>(meta + 4 * kChunk)[col];
  const int sl = reinterpret_cast<const int32_t*>(meta + 8 * kChunk)[col];
  if (!KM_INB(st, sl, k)) return;
  long long* ar = acc + (size_t)r * (k + 1);
  const long long xd = Tr<T>::fx(d, f), xs = Tr<T>::fx(ds, f);
  if (d < dn) {
    const long long xn = Tr<T>::fx(dn, f);
    atomic_add_shared64(ar + k, xd - xn);
    atomic_add_shared64(ar + sl, xn - xs);
  } else {
    atomic_add_shared64(ar + sl, xd - xs);
  }
}

// All hits of one stage for this warp; hmask as above, t = 32 warp + lane.
template <class E>
__device__ __forceinline__ void swap_stage_hits(unsigned long long hmask, uint16_t* q, int lane,
                                                int warp, const E* data,
                                                const unsigned char* meta, long long* acc, int k,
                                                int f, KmState* st) {
  const int cnt = __popcll(hmask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  if (total <= kQueue) {
    int pos = incl - cnt;
    while (hmask) {
      const int b = __ffsll(hmask) - 1;
      hmask &= hmask - 1;
      q[pos++] = (uint16_t)((b << 5) | lane);
    }
    __syncwarp();
    for (int e = lane; e < total; e += 32) {
      const unsigned v = q[e];
      const int b = (int)(v >> 5), src = (int)(v & 31u);
      swap_hit_at<E>(b >> 2, 4 * (warp * 32 + src) + (b & 3), data, meta, acc, k, f, st);
    }
    __syncwarp();
  } else {
    // dense stage (e.g. far-from-converged medoids): every lane its own hits
    while (hmask) {
      const int b = __ffsll(hmask) - 1;
      hmask &= hmask - 1;
      swap_hit_at<E>(b >> 2, 4 * (warp * 32 + lane) + (b & 3), data, meta, acc, k, f, st);
    }
    __syncwarp();
  }
}

template <class E, int MODE, int R, int S, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_stream(const StreamArgs a) {
  using T = typename Val<E>::type;  // value type (16-bit elements widen to int32)
  using G = typename Tr<T>::G;
  using A = long long;  // SWAP accumulators (fixed point / int64)
  using KA = typename std::conditional<MODE == kModeSwap, long long, G>::type;
  using Vec = typename V4<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];

  KmState* st = a.st;
  if (st->done || st->error) return;  // uniform for all CTAs of this launch
  const unsigned long long wlim = wait_limit(st);

  const int n = a.n, m = a.m, k = a.k, f = a.fshift;
  const int fp2 = (MODE == kModeSwap && a.flavour == kFastPAM2);
  const Layout L = make_layout(MODE, R, S, k, fp2, (int)sizeof(E));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  uint64_t* cbar = empty + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.flags);
  volatile int* last_flag = abort_flag + 1;
  int* scratch_int = const_cast<int*>(abort_flag) + 2;
  Key<KA>* wkeys = reinterpret_cast<Key<KA>*>(smem + L.wkeys);
  A* rl = reinterpret_cast<A*>(smem + L.rl);
  G* red = reinterpret_cast<G*>(smem + L.red);
  int* tile_rows = reinterpret_cast<int*>(smem + L.tile_rows);
  A* acc = reinterpret_cast<A*>(smem + L.acc);
  Key<A>* slot_local = reinterpret_cast<Key<A>*>(smem + L.slot_local);
  uint16_t* queues = reinterpret_cast<uint16_t*>(smem + L.queues);
  unsigned char* stages = smem + L.stages;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int rb = st->rb;

  // Block 0 clears the buffers the apply kernel of this pass fills.
  if (MODE == kModeSwap && blockIdx.x == 0 && a.flavour != kEvalOnly) {
    A* rnext = reinterpret_cast<A*>(a.removal) + (size_t)(rb ^ 1) * a.k_pad;
    for (int i = tid; i < k; i += kThreads) rnext[i] = A(0);
    if (tid == 0) reinterpret_cast<G*>(a.td2)[rb ^ 1] = G(0);
  }
  if (MODE == kModeBuild && blockIdx.x == 0 && tid == 0) {
    st->build_td_d = 0.0;
    st->build_td_i = 0;
  }

  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kConsWarps);
    }
    mbar_init(cbar, kConsWarps);
    abort_flag[0] = 0;
    abort_flag[1] = 0;
    fence_barrier_init();
  }
  if (MODE == kModeSwap) {
    const A* rsrc = reinterpret_cast<const A*>(a.removal) + (size_t)rb * a.k_pad;
    for (int i = tid; i < k; i += kThreads) rl[i] = rsrc[i];
    for (int i = tid; i < R * (k + 1); i += kThreads) acc[i] = A(0);
    if (fp2)
      for (int i = tid; i < k; i += kThreads) {
        slot_local[i].d = LLONG_MAX;
        slot_local[i].slot = i;
        slot_local[i].cand = INT_MAX;
      }
  }
  __syncthreads();

  // Candidate positions: a FasterPAM / FastCLARANS window is the next wl
  // scan positions (row = p mod m, or the p-th draw), dealt round-robin so
  // that CTA b takes base + b, base + b + G, ... (G = grid size, at most R
  // each); its length adapts on the device (see the decision below).  Full
  // passes hand out tiles of R rows from an atomic counter so that CTAs on
  // faster paths take more tiles.
  const bool clarans = (MODE == kModeSwap && a.flavour == kCLARANS);
  const bool windowed = (MODE == kModeSwap && (a.flavour == kFasterPAM || clarans));
  const long long wmax = (long long)gridDim.x * a.win_rows;
  long long base = 0, p_lo = 0, p_hi = 0, wl = 0;
  if (windowed) {
    base = st->pos;
    const long long stop =
        clarans ? a.draws_len : ((st->last < 0) ? (long long)m : st->last + m);
    wl = st->win_len;
    if (wl <= 0) wl = gridDim.x;
    if (wl > wmax) wl = wmax;
    p_lo = base + (long long)blockIdx.x;
    p_hi = base + wl;
    if (p_hi > stop) p_hi = stop;
  }
  const unsigned ntiles = (unsigned)((m + R - 1) / R);
  const int nchunks = (n + kChunk - 1) / kChunk;
  // columns copied per row: n rounded up to whole 16-byte pieces
  constexpr int kGran = 16 / (int)sizeof(E);
  const int n4 = (n + kGran - 1) / kGran * kGran;

  // ================================================================ producer
  if (warp == kConsWarps) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      long long p = p_lo;
      bool ok = true;
      uint32_t used = 0, uph = 0;  // stages ever filled, and their parity
      while (ok) {
        int rows[R], outs[R];
        int nr = 0;
        if (windowed) {
          while (nr < R && p < p_hi) {
            const int row = clarans ? a.draws[p] : (int)(p % m);
            if (row >= 0 && row < m && !a.is_med[row]) {
              rows[nr] = row;
              outs[nr] = (int)(p - base);
              ++nr;
            }
            p += gridDim.x;
          }
          if (nr == 0) break;
        } else {
          // next tile with at least one non-medoid row
          while (nr == 0) {
            const unsigned tile = atomicAdd(&st->tile_next, 1u);
            if (tile >= ntiles) break;
            const int r0 = (int)tile * R;
            const int r1 = (r0 + R < m) ? r0 + R : m;
            for (int row = r0; row < r1; ++row)
              if (!a.is_med[row]) {
                rows[nr] = row;
                outs[nr] = row;
                ++nr;
              }
          }
          if (nr == 0) break;
        }
        for (int j = 0; j < nchunks; ++j) {
          if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, wlim)) {
            ok = false;
            break;
          }
          unsigned char* sb = stages + (size_t)s * L.stage_bytes;
          StageHdr* h = reinterpret_cast<StageHdr*>(sb);
          for (int r = 0; r < nr; ++r) {
            h->rows[r] = rows[r];
            h->outidx[r] = outs[r];
          }
          h->nrows = nr;
          h->chunk = j;
          h->first = (j == 0);
          h->last = (j == nchunks - 1);
          const int col0 = j * kChunk;
          const int cols = (n4 - col0 < kChunk) ? (n4 - col0) : kChunk;
          const uint32_t rbytes = (uint32_t)sizeof(E) * (uint32_t)cols;
          const uint32_t mbytes = (uint32_t)L.meta_bytes;
          mbar_arrive_expect_tx(&full[s], rbytes * nr + mbytes);
          used |= 1u << s;
          uph = (uph & ~(1u << s)) | (ph << s);
          unsigned char* meta = sb + 256;
          if (MODE == kModeSwap) {
            bulk_g2s(meta, static_cast<const T*>(a.dn) + col0, 4 * kChunk, &full[s]);
            bulk_g2s(meta + 4 * kChunk, static_cast<const T*>(a.ds) + col0, 4 * kChunk, &full[s]);
            bulk_g2s(meta + 8 * kChunk, a.near + col0, 4 * kChunk, &full[s]);
          } else {
            bulk_g2s(meta, static_cast<const T*>(a.bdn) + col0, 4 * kChunk, &full[s]);
          }
          unsigned char* data = meta + L.meta_bytes;
          const E* D = static_cast<const E*>(a.D);
          for (int r = 0; r < nr; ++r)
            bulk_g2s(data + (size_t)r * sizeof(E) * kChunk, D + (size_t)rows[r] * a.ld + col0,
                     rbytes, &full[s]);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (ok && mbar_wait(&empty[s], ph ^ 1, abort_flag, wlim)) {
        StageHdr* h = reinterpret_cast<StageHdr*>(stages + (size_t)s * L.stage_bytes);
        h->nrows = 0;
        mbar_arrive(&full[s]);
      } else {
        abort_flag[0] = 1;
        atomicExch(&st->error, kErrTimeout);
        // let every copy already issued land before the CTA may exit
        volatile int never = 0;
        for (int q = 0; q < S; ++q)
          if (used & (1u << q)) (void)mbar_wait(&full[q], (uph >> q) & 1u, &never);
      }
    }
    return;
  }

  // ================================================================ consumers
  const int t = tid;  // 0..255, owns columns 4t..4t+3 of each chunk
  Key<KA> wbest;
  wbest.d = (MODE == kModeSwap) ? KA(LLONG_MAX) : KA(Tr<T>::g_high());
  wbest.slot = INT_MAX;
  wbest.cand = INT_MAX;

  // BUILD per-row partial sums (registers): compensated FP32 or int64
  float ks[R], kc[R];
  long long ki[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    ks[r] = 0.f;
    kc[r] = 0.f;
    ki[r] = 0;
  }

  uint32_t cph = 0;  // consumer barrier phase
#define KM_CSYNC()                              \
  do {                                          \
    if (!cons_sync(cbar, cph, abort_flag, wlim)) {\
      abort_flag[0] = 1;                        \
      atomicExch(&st->error, kErrTimeout);      \
      return;                                   \
    }                                           \
  } while (0)
  int s = 0;
  uint32_t ph = 0;
  while (true) {
    if (!mbar_wait(&full[s], ph, abort_flag, wlim)) {
      abort_flag[0] = 1;
      atomicExch(&st->error, kErrTimeout);
      return;
    }
    const unsigned char* sb = stages + (size_t)s * L.stage_bytes;
    const StageHdr* h = reinterpret_cast<const StageHdr*>(sb);
    const int nr = h->nrows;
    if (nr == 0) break;
    const int chunk = h->chunk;
    const int is_last = h->last;
    const int my_row = (lane < nr) ? h->rows[lane] : -1;
    const int my_out = (lane < nr) ? h->outidx[lane] : -1;
    const unsigned char* meta = sb + 256;
    const E* data = reinterpret_cast<const E*>(meta + L.meta_bytes);

    if (MODE == kModeSwap) {
      const Vec ds4 = lds4(reinterpret_cast<const T*>(meta + 4 * kChunk) + 4 * t);
      unsigned long long hmask = 0ull;
#pragma unroll 4
      for (int r = 0; r < nr; ++r) {
        const Vec d4 = ld4e(data + (size_t)r * kChunk + 4 * t);
        const unsigned hm = (d4.x < ds4.x ? 1u : 0u) | (d4.y < ds4.y ? 2u : 0u) |
                            (d4.z < ds4.z ? 4u : 0u) | (d4.w < ds4.w ? 8u : 0u);
        hmask |= (unsigned long long)hm << (4 * r);
      }
      swap_stage_hits<E>(hmask, queues + warp * kQueue, lane, warp, data, meta, acc, k, f, st);
    } else {
      const int col = chunk * kChunk + 4 * t;
      const bool v0 = col < n, v1 = col + 1 < n, v2 = col + 2 < n, v3 = col + 3 < n;
      const Vec dn4 = lds4(reinterpret_cast<const T*>(meta) + 4 * t);
      const bool first = a.build_first != 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < nr) {
          const Vec d4 = ld4e(data + (size_t)r * kChunk + 4 * t);
          T x0, x1, x2, x3;
          if (first) {
            x0 = v0 ? d4.x : T(0);
            x1 = v1 ? d4.y : T(0);
            x2 = v2 ? d4.z : T(0);
            x3 = v3 ? d4.w : T(0);
          } else {
            // padding columns carry the lowest sentinel: never below it
            x0 = (d4.x < dn4.x) ? T(d4.x - dn4.x) : T(0);
            x1 = (d4.y < dn4.y) ? T(d4.y - dn4.y) : T(0);
            x2 = (d4.z < dn4.z) ? T(d4.z - dn4.z) : T(0);
            x3 = (d4.w < dn4.w) ? T(d4.w - dn4.w) : T(0);
          }
          if constexpr (std::is_same<T, float>::value) {
            // the four terms share a sign: their FP32 sum is within 2 ulp;
            // the row sum is then carried with Kahan compensation
            const float p4 = (x0 + x1) + (x2 + x3);
            const float y = p4 - kc[r];
            const float tt = ks[r] + y;
            kc[r] = (tt - ks[r]) - y;
            ks[r] = tt;
          } else {
            ki[r] += (long long)x0 + (long long)x1 + (long long)x2 + (long long)x3;
          }
        }
      }
    }

    // release the stage
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (++s == S) {
      s = 0;
      ph ^= 1;
    }

    if (!is_last) continue;

    // ------------------------------------------------------ tile finished
    if (MODE == kModeSwap) {
      if (warp == 0 && lane < nr) tile_rows[lane] = my_row;
      KM_CSYNC();
      for (int r = warp; r < nr; r += kConsWarps) {
        const A* ar = acc + (size_t)r * (k + 1);
        Key<A> kb;
        kb.d = LLONG_MAX;
        kb.slot = INT_MAX;
        kb.cand = 0;
        for (int i = lane; i < k; i += 32) {
          const A v = rl[i] + ar[i];
          if (v < kb.d) {
            kb.d = v;
            kb.slot = i;
          }
        }
        kb = warp_min_key(kb);
        const A total = kb.d + ar[k];
        const int c = __shfl_sync(0xffffffffu, my_row, r);
        const int out = __shfl_sync(0xffffffffu, my_out, r);
        if (lane == 0) {
          if (a.cand_delta) a.cand_delta[out] = Tr<T>::unfx(total, f);
          if (a.cand_slot) a.cand_slot[out] = kb.slot;
          Key<KA> ck;
          ck.d = total;
          ck.slot = kb.slot;
          ck.cand = c;
          if (key_less(ck, wbest)) wbest = ck;
        }
      }
      if (fp2) {
        for (int i = t; i < k; i += kConsThreads) {
          Key<A> sbk = slot_local[i];
          for (int r = 0; r < nr; ++r) {
            const A* ar = acc + (size_t)r * (k + 1);
            const A v = (rl[i] + ar[i]) + ar[k];
            const int c = tile_rows[r];
            if (v < sbk.d || (v == sbk.d && c < sbk.cand)) {
              sbk.d = v;
              sbk.cand = c;
            }
          }
          slot_local[i] = sbk;
        }
      }
      KM_CSYNC();
      for (int e = t; e < nr * (k + 1); e += kConsThreads) acc[e] = A(0);
      KM_CSYNC();
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (std::is_same<T, float>::value) {
          // value = hi + lo (Kahan keeps sum - compensation); add across the
          // warp with error-free TwoSum in FP32, one FP64 fold per row
          float hi = ks[r], lo = -kc[r];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
            const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
            const float sh = hi + ohi;
            const float bp = sh - hi;
            const float err = (hi - (sh - bp)) + (ohi - bp);
            hi = sh;
            lo = lo + olo + err;
          }
          if (lane == 0) red[warp * R + r] = (double)hi + (double)lo;
        } else {
          const long long v = warp_sum(ki[r]);
          if (lane == 0) red[warp * R + r] = v;
        }
        ks[r] = 0.f;
        kc[r] = 0.f;
        ki[r] = 0;
      }
      KM_CSYNC();
      if (warp == 0) {
        Key<KA> kb;
        kb.d = Tr<T>::g_high();
        kb.slot = 0;
        kb.cand = INT_MAX;
        if (lane < nr) {
          G tot = G(0);
          for (int w = 0; w < kConsWarps; ++w) tot += red[w * R + lane];
          kb.d = tot;
          kb.cand = my_row;
          if (a.cand_gain) a.cand_gain[my_out] = to_double(tot);
        }
        kb = warp_min_key(kb);
        if (lane == 0 && key_less(kb, wbest)) wbest = kb;
      }
      KM_CSYNC();
    }
  }

  // ------------------------------------------------------------ CTA result
  if (lane == 0) wkeys[warp] = wbest;
  if (fp2) {
    Key<A>* sp = reinterpret_cast<Key<A>*>(a.slot_partials) + (size_t)blockIdx.x * k;
    for (int i = t; i < k; i += kConsThreads) sp[i] = slot_local[i];
  }
  __threadfence();
  KM_CSYNC();
  if (t == 0) {
    Key<KA> b = wkeys[0];
    for (int w = 1; w < kConsWarps; ++w)
      if (key_less(wkeys[w], b)) b = wkeys[w];
    reinterpret_cast<Key<KA>*>(a.partials)[blockIdx.x] = b;
    __threadfence();
    const unsigned tk = atomicAdd(&st->ticket, 1u);
    last_flag[0] = (tk == gridDim.x - 1) ? 1 : 0;
  }
  KM_CSYNC();
  if (!last_flag[0]) return;

  // ------------------------------------------------- last CTA: grid result
  __threadfence();
  const Key<KA>* parts = reinterpret_cast<const Key<KA>*>(a.partials);
  if (warp == 0) {
    Key<KA> b;
    b.d = (MODE == kModeSwap) ? KA(LLONG_MAX) : KA(Tr<T>::g_high());
    b.slot = INT_MAX;
    b.cand = INT_MAX;
    for (int g = lane; g < (int)gridDim.x; g += 32) {
      const Key<KA> v = ld_cg_key(parts + g);
      if (key_less(v, b)) b = v;
    }
    b = warp_min_key(b);
    if (lane == 0) wkeys[0] = b;
  }
  KM_CSYNC();
  const Key<KA> best = wkeys[0];

  if (MODE == kModeBuild) {
    if (t == 0) {
      st->build_gain_d = to_double(best.d);
      st->build_gain_i = (long long)best.d;
      st->build_cand = best.cand;
      st->tile_next = 0;
      st->ticket = 0;
    }
    return;
  }

  if (clarans) {
    // FastCLARANS: the first improving draw of the window, in draw order,
    // unless maxneighbor consecutive draws fail before it (Sec. 3.4)
    const long long stop = a.draws_len;
    long long wlen = wl;
    if (base + wlen > stop) wlen = stop - base;
    int* firstw = scratch_int;
    int* nfail = scratch_int + 1;
    if (t == 0) {
      *firstw = INT_MAX;
      *nfail = 0;
    }
    KM_CSYNC();
    for (long long w = t; w < wlen; w += kConsThreads) {
      const int row = a.draws[base + w];
      if (row < 0 || row >= m || a.is_med[row]) continue;
      if (__ldcg(a.cand_slot + w) >= 0 && __ldcg(a.cand_delta + w) < -a.tol)
        atomicMin(firstw, (int)w);
    }
    KM_CSYNC();
    const int fw = *firstw;
    int cnt = 0;  // evaluated draws before the first improving one
    for (long long w = t; w < wlen && w < fw; w += kConsThreads) {
      const int row = a.draws[base + w];
      if (row >= 0 && row < m && !a.is_med[row]) ++cnt;
    }
    if (cnt) atomicAdd(nfail, cnt);
    KM_CSYNC();
    if (t == 0) {
      const long long F = *nfail;
      if (st->fails + F >= a.maxneighbor) {
        // stop at the draw that makes the failure count reach maxneighbor
        const long long need = a.maxneighbor - st->fails;
        long long seen = 0, w = 0;
        for (; w < wlen; ++w) {
          const int row = a.draws[base + w];
          if (row >= 0 && row < m && !a.is_med[row] && ++seen == need) break;
        }
        st->accept = 0;
        st->done = 1;
        st->fails = a.maxneighbor;
        st->evaluated += need;
        st->pos = base + w + 1;
      } else if (fw != INT_MAX) {
        const double dw = __ldcg(a.cand_delta + fw);
        st->accept = 1;
        st->best_d = dw;
        st->best_i = (long long)dw;
        st->best_slot = __ldcg(a.cand_slot + fw);
        st->best_cand = a.draws[base + fw];
        st->fails = 0;
        st->evaluated += F + 1;
        st->last = base + fw;
        st->pos = base + fw + 1;
        st->win_len = gridDim.x;
      } else {
        st->accept = 0;
        st->fails += F;
        st->evaluated += F;
        st->pos = base + wlen;
        if (st->pos >= stop) st->done = 1;
        st->win_len = (2 * wl < wmax) ? 2 * wl : wmax;
      }
      st->iter += 1;
      st->ticket = 0;
    }
    return;
  }

  // Window length of the next launch: one position per CTA after a swap
  // (swaps are then frequent, and a window of G rows costs little more than
  // the launch), doubled up to G R after a window without one (a converged
  // scan then streams at full bandwidth).  The decisions do not depend on
  // the window length: positions after the first improving one are
  // evaluated again against the new state.
  if (a.flavour == kFasterPAM) {
    // first improving candidate of the window, in scan order
    const long long stop = (st->last < 0) ? (long long)m : st->last + m;
    long long wlen = wl;
    if (base + wlen > stop) wlen = stop - base;
    int* firstw = scratch_int;
    int* nev = scratch_int + 1;
    if (t == 0) {
      *firstw = INT_MAX;
      *nev = 0;
    }
    KM_CSYNC();
    for (long long w = t; w < wlen; w += kConsThreads) {
      const int row = (int)((base + w) % m);
      if (a.is_med[row]) continue;
      if (__ldcg(a.cand_slot + w) >= 0 && __ldcg(a.cand_delta + w) < -a.tol)
        atomicMin(firstw, (int)w);
    }
    KM_CSYNC();
    {
      // evaluated (non-medoid) positions up to and including the first
      // improving one
      const int fw0 = *firstw;
      int cnt = 0;
      for (long long w = t; w < wlen && w <= fw0; w += kConsThreads)
        if (!a.is_med[(int)((base + w) % m)]) ++cnt;
      if (cnt) atomicAdd(nev, cnt);
    }
    KM_CSYNC();
    if (t == 0) {
      const int w = *firstw;
      st->evaluated += *nev;
      if (w != INT_MAX) {
        const double dw = __ldcg(a.cand_delta + w);
        st->accept = 1;
        st->best_d = dw;
        st->best_i = (long long)dw;
        st->best_slot = __ldcg(a.cand_slot + w);
        st->best_cand = (int)((base + w) % m);
        st->last = base + w;
        st->pos = base + w + 1;
        st->win_len = gridDim.x;
      } else {
        st->accept = 0;
        st->pos = base + wlen;
        if (st->pos >= stop) st->done = 1;
        st->win_len = (2 * wl < wmax) ? 2 * wl : wmax;
      }
      st->iter += 1;
      st->ticket = 0;
    }
    return;
  }

  if (t == 0) {
    const double bd = Tr<T>::unfx((long long)best.d, f);
    st->best_d = bd;
    st->best_i = (long long)best.d;
    st->best_slot = (best.cand == INT_MAX) ? -1 : best.slot;
    st->best_cand = (best.cand == INT_MAX) ? -1 : best.cand;
    if (a.flavour != kEvalOnly) {
      st->iter += 1;
      if (best.cand != INT_MAX && bd < -a.tol) {
        st->accept = 1;
      } else {
        st->accept = 0;
        st->done = 1;
      }
    }
  }
  if (fp2) {
    // per-slot best over the grid, then the queue of additional swaps
    Key<A>* sbest = reinterpret_cast<Key<A>*>(a.slot_best);
    const Key<A>* sp = reinterpret_cast<const Key<A>*>(a.slot_partials);
    for (int i = t; i < k; i += kConsThreads) {
      Key<A> b = ld_cg_key(sp + i);
      for (int g = 1; g < (int)gridDim.x; ++g) {
        const Key<A> v = ld_cg_key(sp + (size_t)g * k + i);
        if (v.d < b.d || (v.d == b.d && v.cand < b.cand)) b = v;
      }
      sbest[i] = b;
    }
    __threadfence_block();
    KM_CSYNC();
    const int bslot = (best.cand == INT_MAX) ? -1 : best.slot;
    int* cnt = scratch_int;
    if (t == 0) *cnt = 0;
    KM_CSYNC();
    for (int i = t; i < k; i += kConsThreads) {
      const Key<A> ki2 = sbest[i];
      const bool elig = (i != bslot) && ki2.cand != INT_MAX && ki2.d < 0;
      if (!elig) continue;
      int rank = 0;
      for (int j = 0; j < k; ++j) {
        if (j == i || j == bslot) continue;
        const Key<A> kj = sbest[j];
        if (!(kj.cand != INT_MAX && kj.d < 0)) continue;
        if (kj.d < ki2.d || (kj.d == ki2.d && j < i)) ++rank;
      }
      a.fp2_order[rank] = i;
      atomicAdd(cnt, 1);
    }
    KM_CSYNC();
    if (t == 0) {
      st->fp2_extra = (st->accept) ? *cnt : 0;
      st->fp2_dstar = fabs(Tr<T>::unfx((long long)best.d, f));
    }
  }
  if (t == 0) {
    st->tile_next = 0;
    st->ticket = 0;
  }
#undef KM_CSYNC
}

// ------------------------------------------------------------- host side
// Kernel geometries: rows per tile (= per stage), ring stages, CTAs per SM.
struct Geometry {
  int rows, stages, minb;
};
static const Geometry kGeoms[] = {
    {16, 2, 1},  // 1
    {8, 4, 1},   // 2
    {8, 2, 2},   // 3
    {4, 4, 1},   // 4
    {2, 4, 1},   // 5
    {1, 4, 1},   // 6
    {16, 3, 1},  // 7
    {8, 5, 1},   // 8
    {4, 2, 2},   // 9
    {4, 3, 2},   // 10
    {4, 2, 3},   // 11
    {8, 2, 3},   // 12
    {2, 3, 3},   // 13
    {4, 3, 3},   // 14
    {8, 3, 2},   // 15
    {2, 4, 3},   // 16
};
static const int kNumGeoms = sizeof(kGeoms) / sizeof(kGeoms[0]);

bool stream_config(int mode, int k, int flavour, int forced_rows, int tune, StreamConfig* cfg,
                   int esize) {
  const int fp2 = (mode == kModeSwap && flavour == kFastPAM2);
  auto fits = [&](const Geometry& g, size_t* bytes) {
    const Layout L = make_layout(mode, g.rows, g.stages, k, fp2, esize);
    const size_t limit = (size_t)228 * 1024 / g.minb - 1024;
    *bytes = L.total;
    return L.total <= limit;
  };
  if (tune > 0) {
    if (tune > kNumGeoms) return false;
    const Geometry& g = kGeoms[tune - 1];
    size_t b;
    if (!fits(g, &b)) return false;
    *cfg = {g.rows, g.stages, g.minb, b, tune};
    return true;
  }
  // automatic: the first geometry of the preference list that fits.  The
  // order comes from sweeps on GB300 (n = 20000 and 50000 float matrices):
  // BUILD streams best with 3 CTAs/SM of 4-row tiles and a 3-stage ring;
  // SWAP with 2 CTAs/SM of 8-row tiles (its shared accumulators grow with
  // k, so larger k falls back to smaller footprints).
  static const int pref_swap[] = {3, 11, 1, 2, 4, 5, 6};
  static const int pref_build[] = {14, 12, 15, 3, 11, 1, 2, 4, 5, 6};
  const int* pref = (mode == kModeSwap) ? pref_swap : pref_build;
  const int npref = (mode == kModeSwap) ? 7 : 10;
  for (int q = 0; q < npref; ++q) {
    const Geometry& g = kGeoms[pref[q] - 1];
    if (forced_rows > 0 && g.rows != forced_rows) continue;
    size_t b;
    if (fits(g, &b)) {
      *cfg = {g.rows, g.stages, g.minb, b, pref[q]};
      return true;
    }
  }
  return false;
}

template <class E, int MODE, int R, int S, int MINB>
static cudaError_t launch_one(const StreamConfig& cfg, int grid, const StreamArgs& a,
                              cudaStream_t s) {
  auto kern = k_stream<E, MODE, R, S, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cfg.smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, cfg.smem, s>>>(a);
  return cudaGetLastError();
}

template <class T, int MODE>
static cudaError_t launch_geo(const StreamConfig& cfg, int grid, const StreamArgs& a,
                              cudaStream_t s) {
  switch (cfg.geometry) {
    case 1: return launch_one<T, MODE, 16, 2, 1>(cfg, grid, a, s);
    case 2: return launch_one<T, MODE, 8, 4, 1>(cfg, grid, a, s);
    case 3: return launch_one<T, MODE, 8, 2, 2>(cfg, grid, a, s);
    case 4: return launch_one<T, MODE, 4, 4, 1>(cfg, grid, a, s);
    case 5: return launch_one<T, MODE, 2, 4, 1>(cfg, grid, a, s);
    case 6: return launch_one<T, MODE, 1, 4, 1>(cfg, grid, a, s);
    case 7: return launch_one<T, MODE, 16, 3, 1>(cfg, grid, a, s);
    case 8: return launch_one<T, MODE, 8, 5, 1>(cfg, grid, a, s);
    case 9: return launch_one<T, MODE, 4, 2, 2>(cfg, grid, a, s);
    case 10: return launch_one<T, MODE, 4, 3, 2>(cfg, grid, a, s);
    case 11: return launch_one<T, MODE, 4, 2, 3>(cfg, grid, a, s);
    case 12: return launch_one<T, MODE, 8, 2, 3>(cfg, grid, a, s);
    case 13: return launch_one<T, MODE, 2, 3, 3>(cfg, grid, a, s);
    case 14: return launch_one<T, MODE, 4, 3, 3>(cfg, grid, a, s);
    case 15: return launch_one<T, MODE, 8, 3, 2>(cfg, grid, a, s);
    case 16: return launch_one<T, MODE, 2, 4, 3>(cfg, grid, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stream(int dtype, int mode, const StreamConfig& cfg, int grid,
                          const StreamArgs& a, cudaStream_t s) {
  if (dtype == 0)
    return mode == kModeSwap ? launch_geo<int32_t, kModeSwap>(cfg, grid, a, s)
                             : launch_geo<int32_t, kModeBuild>(cfg, grid, a, s);
  if (dtype == 2)
    return mode == kModeSwap ? launch_geo<uint16_t, kModeSwap>(cfg, grid, a, s)
                             : launch_geo<uint16_t, kModeBuild>(cfg, grid, a, s);
  return mode == kModeSwap ? launch_geo<float, kModeSwap>(cfg, grid, a, s)
                           : launch_geo<float, kModeBuild>(cfg, grid, a, s);
}

}  // namespace km

extern "C" int kmedoids_geometry_info(int32_t geometry, int32_t* rows, int32_t* stages,
                                      int32_t* ctas_per_sm) {
  if (geometry < 1 || geometry > km::kNumGeoms) return 1;
  const km::Geometry& g = km::kGeoms[geometry - 1];
  if (rows) *rows = g.rows;
  if (stages) *stages = g.stages;
  if (ctas_per_sm) *ctas_per_sm = g.minb;
  return 0;
}

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

struct Layout {
  size_t bars, flags, wkeys, rl, red, tile_rows, acc, slot_local, stages;
  size_t stage_bytes, meta_bytes, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Offsets of the dynamic shared-memory regions (bytes).
__host__ __device__ inline Layout make_layout(int mode, int R, int S, int k, int fp2) {
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
  o = align_up(o, 128);
  L.stages = o;
  L.meta_bytes = (mode == kModeSwap) ? 3 * 4 * (size_t)kChunk : 4 * (size_t)kChunk;
  L.stage_bytes = 256 + L.meta_bytes + 4 * (size_t)R * kChunk;
  o += L.stage_bytes * S;
  L.total = o;
  return L;
}

// --------------------------------------------------------------- kernel
template <class T, int MODE, int R, int S>
__global__ void __launch_bounds__(kThreads, 1) k_stream(const StreamArgs a) {
  using A = typename Tr<T>::A;
  using Vec = typename V4<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];

  KmState* st = a.st;
  if (st->done || st->error) return;  // uniform for all CTAs of this launch

  const int n = a.n, k = a.k;
  const int fp2 = (MODE == kModeSwap && a.flavour == kFastPAM2);
  const Layout L = make_layout(MODE, R, S, k, fp2);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  uint64_t* cbar = empty + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.flags);
  volatile int* last_flag = abort_flag + 1;
  Key<A>* wkeys = reinterpret_cast<Key<A>*>(smem + L.wkeys);
  A* rl = reinterpret_cast<A*>(smem + L.rl);
  double* red = reinterpret_cast<double*>(smem + L.red);
  int* tile_rows = reinterpret_cast<int*>(smem + L.tile_rows);
  A* acc = reinterpret_cast<A*>(smem + L.acc);
  Key<A>* slot_local = reinterpret_cast<Key<A>*>(smem + L.slot_local);
  unsigned char* stages = smem + L.stages;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int rb = st->rb;

  // Block 0 clears the buffers the apply kernel of this pass fills.
  if (MODE == kModeSwap && blockIdx.x == 0 && a.flavour != kEvalOnly) {
    A* rnext = reinterpret_cast<A*>(a.removal) + (size_t)(rb ^ 1) * a.k_pad;
    for (int i = tid; i < k; i += kThreads) rnext[i] = A(0);
    if (tid == 0) reinterpret_cast<A*>(a.td2)[rb ^ 1] = A(0);
  }
  if (MODE == kModeBuild && blockIdx.x == 0 && tid == 0) {
    st->build_td_d = 0.0;
    st->build_td_i = 0;
  }

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsWarps);
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
        slot_local[i].d = Tr<T>::a_high();
        slot_local[i].slot = i;
        slot_local[i].cand = INT_MAX;
      }
  }
  __syncthreads();

  // Candidate positions of this CTA: [p_lo, p_hi); row = p mod n.
  long long base = 0, p_lo, p_hi;
  if (MODE == kModeSwap && a.flavour == kFasterPAM) {
    base = st->pos;
    const long long stop = (st->last < 0) ? (long long)n : st->last + n;
    p_lo = base + (long long)blockIdx.x * a.win_rows;
    p_hi = p_lo + a.win_rows;
    if (p_hi > stop) p_hi = stop;
  } else {
    p_lo = (long long)blockIdx.x * n / gridDim.x;
    p_hi = (long long)(blockIdx.x + 1) * n / gridDim.x;
  }
  const int nchunks = (n + kChunk - 1) / kChunk;
  const int n4 = (n + 3) & ~3;

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
        while (nr < R && p < p_hi) {
          const int row = (int)(p % n);
          if (!a.is_med[row]) {
            rows[nr] = row;
            outs[nr] = (int)(p - base);
            ++nr;
          }
          ++p;
        }
        if (nr == 0) break;
        for (int j = 0; j < nchunks; ++j) {
          if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
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
          const uint32_t rbytes = 4u * (uint32_t)cols;
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
          const T* D = static_cast<const T*>(a.D);
          for (int r = 0; r < nr; ++r)
            bulk_g2s(data + (size_t)r * 4 * kChunk, D + (size_t)rows[r] * a.ld + col0, rbytes,
                     &full[s]);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (ok && mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
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
  Key<A> wbest;
  wbest.d = Tr<T>::a_high();
  wbest.slot = INT_MAX;
  wbest.cand = INT_MAX;

  // BUILD per-row partial sums (registers)
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
    if (!cons_sync(cbar, cph, abort_flag)) {    \
      abort_flag[0] = 1;                        \
      atomicExch(&st->error, kErrTimeout);      \
      return;                                   \
    }                                           \
  } while (0)
  int s = 0;
  uint32_t ph = 0;
  while (true) {
    if (!mbar_wait(&full[s], ph, abort_flag)) {
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
    const T* data = reinterpret_cast<const T*>(meta + L.meta_bytes);

    if (MODE == kModeSwap) {
      const Vec dn4 = lds4(reinterpret_cast<const T*>(meta) + 4 * t);
      const Vec ds4 = lds4(reinterpret_cast<const T*>(meta + 4 * kChunk) + 4 * t);
      const int4 nr4 = lds4(reinterpret_cast<const int32_t*>(meta + 8 * kChunk) + 4 * t);
#pragma unroll 4
      for (int r = 0; r < nr; ++r) {
        const Vec d4 = lds4(data + (size_t)r * kChunk + 4 * t);
        const bool h0 = d4.x < ds4.x, h1 = d4.y < ds4.y, h2 = d4.z < ds4.z, h3 = d4.w < ds4.w;
        if (h0 | h1 | h2 | h3) {
          A* ar = acc + (size_t)r * (k + 1);
          if (h0) {
            if (d4.x < dn4.x) {
              atomic_add_acc(ar + k, dif(d4.x, dn4.x));
              atomic_add_acc(ar + nr4.x, dif(dn4.x, ds4.x));
            } else {
              atomic_add_acc(ar + nr4.x, dif(d4.x, ds4.x));
            }
          }
          if (h1) {
            if (d4.y < dn4.y) {
              atomic_add_acc(ar + k, dif(d4.y, dn4.y));
              atomic_add_acc(ar + nr4.y, dif(dn4.y, ds4.y));
            } else {
              atomic_add_acc(ar + nr4.y, dif(d4.y, ds4.y));
            }
          }
          if (h2) {
            if (d4.z < dn4.z) {
              atomic_add_acc(ar + k, dif(d4.z, dn4.z));
              atomic_add_acc(ar + nr4.z, dif(dn4.z, ds4.z));
            } else {
              atomic_add_acc(ar + nr4.z, dif(d4.z, ds4.z));
            }
          }
          if (h3) {
            if (d4.w < dn4.w) {
              atomic_add_acc(ar + k, dif(d4.w, dn4.w));
              atomic_add_acc(ar + nr4.w, dif(dn4.w, ds4.w));
            } else {
              atomic_add_acc(ar + nr4.w, dif(d4.w, ds4.w));
            }
          }
        }
      }
    } else {
      const int col = chunk * kChunk + 4 * t;
      const bool v0 = col < n, v1 = col + 1 < n, v2 = col + 2 < n, v3 = col + 3 < n;
      const Vec dn4 = lds4(reinterpret_cast<const T*>(meta) + 4 * t);
      const bool first = a.build_first != 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < nr) {
          const Vec d4 = lds4(data + (size_t)r * kChunk + 4 * t);
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
          if constexpr (sizeof(A) == 8 && std::is_same<T, float>::value) {
            // compensated (Kahan) FP32 partial sums, folded into FP64 per tile
            float y, tt;
            y = float(x0) - kc[r]; tt = ks[r] + y; kc[r] = (tt - ks[r]) - y; ks[r] = tt;
            y = float(x1) - kc[r]; tt = ks[r] + y; kc[r] = (tt - ks[r]) - y; ks[r] = tt;
            y = float(x2) - kc[r]; tt = ks[r] + y; kc[r] = (tt - ks[r]) - y; ks[r] = tt;
            y = float(x3) - kc[r]; tt = ks[r] + y; kc[r] = (tt - ks[r]) - y; ks[r] = tt;
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
        kb.d = Tr<T>::a_high();
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
          if (a.cand_delta) a.cand_delta[out] = to_double(total);
          if (a.cand_slot) a.cand_slot[out] = kb.slot;
          Key<A> ck;
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
        double v;
        if constexpr (std::is_same<T, float>::value) {
          v = (double)ks[r] - (double)kc[r];
        } else {
          v = 0.0;
        }
        long long vi = ki[r];
        if constexpr (std::is_same<T, float>::value) {
          v = warp_sum(v);
          if (lane == 0) red[warp * R + r] = v;
        } else {
          vi = warp_sum(vi);
          if (lane == 0) reinterpret_cast<long long*>(red)[warp * R + r] = vi;
        }
        ks[r] = 0.f;
        kc[r] = 0.f;
        ki[r] = 0;
      }
      KM_CSYNC();
      if (warp == 0) {
        Key<A> kb;
        kb.d = Tr<T>::a_high();
        kb.slot = 0;
        kb.cand = INT_MAX;
        if (lane < nr) {
          A tot = A(0);
          for (int w = 0; w < kConsWarps; ++w) {
            if constexpr (std::is_same<T, float>::value)
              tot += red[w * R + lane];
            else
              tot += reinterpret_cast<const long long*>(red)[w * R + lane];
          }
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
    Key<A> b = wkeys[0];
    for (int w = 1; w < kConsWarps; ++w)
      if (key_less(wkeys[w], b)) b = wkeys[w];
    reinterpret_cast<Key<A>*>(a.partials)[blockIdx.x] = b;
    __threadfence();
    const unsigned tk = atomicAdd(&st->ticket, 1u);
    last_flag[0] = (tk == gridDim.x - 1) ? 1 : 0;
  }
  KM_CSYNC();
  if (!last_flag[0]) return;

  // ------------------------------------------------- last CTA: grid result
  __threadfence();
  const Key<A>* parts = reinterpret_cast<const Key<A>*>(a.partials);
  if (warp == 0) {
    Key<A> b;
    b.d = Tr<T>::a_high();
    b.slot = INT_MAX;
    b.cand = INT_MAX;
    for (int g = lane; g < (int)gridDim.x; g += 32) {
      const Key<A> v = ld_cg_key(parts + g);
      if (key_less(v, b)) b = v;
    }
    b = warp_min_key(b);
    if (lane == 0) wkeys[0] = b;
  }
  KM_CSYNC();
  const Key<A> best = wkeys[0];

  if (MODE == kModeBuild) {
    if (t == 0) {
      st->build_gain_d = to_double(best.d);
      st->build_gain_i = (long long)best.d;
      st->build_cand = best.cand;
      st->ticket = 0;
    }
    return;
  }

  if (a.flavour == kFasterPAM) {
    // first improving candidate of the window, in scan order
    const long long stop = (st->last < 0) ? (long long)n : st->last + n;
    long long wlen = (long long)gridDim.x * a.win_rows;
    if (base + wlen > stop) wlen = stop - base;
    int* firstw = const_cast<int*>(last_flag) + 1;
    if (t == 0) *firstw = INT_MAX;
    KM_CSYNC();
    for (long long w = t; w < wlen; w += kConsThreads) {
      const int row = (int)((base + w) % n);
      if (a.is_med[row]) continue;
      if (__ldcg(a.cand_slot + w) >= 0 && __ldcg(a.cand_delta + w) < -a.tol)
        atomicMin(firstw, (int)w);
    }
    KM_CSYNC();
    if (t == 0) {
      const int w = *firstw;
      if (w != INT_MAX) {
        st->accept = 1;
        const double dw = __ldcg(a.cand_delta + w);
        st->best_d = dw;
        st->best_i = (long long)dw;
        st->best_slot = __ldcg(a.cand_slot + w);
        st->best_cand = (int)((base + w) % n);
        st->last = base + w;
        st->pos = base + w + 1;
      } else {
        st->accept = 0;
        st->pos = base + wlen;
        if (st->pos >= stop) st->done = 1;
      }
      st->iter += 1;
      st->ticket = 0;
    }
    return;
  }

  if (t == 0) {
    st->best_d = to_double(best.d);
    st->best_i = (long long)best.d;
    st->best_slot = (best.cand == INT_MAX) ? -1 : best.slot;
    st->best_cand = (best.cand == INT_MAX) ? -1 : best.cand;
    if (a.flavour != kEvalOnly) {
      st->iter += 1;
      if (best.cand != INT_MAX && to_double(best.d) < -a.tol) {
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
    int* cnt = const_cast<int*>(last_flag) + 1;
    if (t == 0) *cnt = 0;
    KM_CSYNC();
    for (int i = t; i < k; i += kConsThreads) {
      const Key<A> ki2 = sbest[i];
      const bool elig = (i != bslot) && ki2.cand != INT_MAX && to_double(ki2.d) < 0.0;
      if (!elig) continue;
      int rank = 0;
      for (int j = 0; j < k; ++j) {
        if (j == i || j == bslot) continue;
        const Key<A> kj = sbest[j];
        if (!(kj.cand != INT_MAX && to_double(kj.d) < 0.0)) continue;
        if (kj.d < ki2.d || (kj.d == ki2.d && j < i)) ++rank;
      }
      a.fp2_order[rank] = i;
      atomicAdd(cnt, 1);
    }
    KM_CSYNC();
    if (t == 0) {
      st->fp2_extra = (st->accept) ? *cnt : 0;
      st->fp2_dstar = fabs(to_double(best.d));
      st->fp2_dstar_i = (best.d < A(0)) ? -(long long)best.d : (long long)best.d;
    }
  }
  if (t == 0) st->ticket = 0;
#undef KM_CSYNC
}

// ------------------------------------------------------------- host side
bool stream_config(int mode, int k, int flavour, int forced_rows, StreamConfig* cfg) {
  static const int cand[][2] = {{16, 2}, {8, 3}, {4, 4}, {2, 4}, {1, 4}};
  const size_t limit = 227 * 1024;
  const int fp2 = (mode == kModeSwap && flavour == kFastPAM2);
  for (auto& rs : cand) {
    if (forced_rows > 0 && rs[0] != forced_rows) continue;
    const Layout L = make_layout(mode, rs[0], rs[1], k, fp2);
    if (L.total <= limit) {
      cfg->rows = rs[0];
      cfg->stages = rs[1];
      cfg->smem = L.total;
      return true;
    }
  }
  return false;
}

template <class T, int MODE, int R, int S>
static cudaError_t launch_one(const StreamConfig& cfg, int grid, const StreamArgs& a,
                              cudaStream_t s) {
  auto kern = k_stream<T, MODE, R, S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cfg.smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, cfg.smem, s>>>(a);
  return cudaGetLastError();
}

template <class T, int MODE>
static cudaError_t launch_rs(const StreamConfig& cfg, int grid, const StreamArgs& a,
                             cudaStream_t s) {
  switch (cfg.rows) {
    case 16:
      return launch_one<T, MODE, 16, 2>(cfg, grid, a, s);
    case 8:
      return launch_one<T, MODE, 8, 3>(cfg, grid, a, s);
    case 4:
      return launch_one<T, MODE, 4, 4>(cfg, grid, a, s);
    case 2:
      return launch_one<T, MODE, 2, 4>(cfg, grid, a, s);
    case 1:
      return launch_one<T, MODE, 1, 4>(cfg, grid, a, s);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stream(int dtype, int mode, const StreamConfig& cfg, int grid,
                          const StreamArgs& a, cudaStream_t s) {
  if (dtype == 0)
    return mode == kModeSwap ? launch_rs<int32_t, kModeSwap>(cfg, grid, a, s)
                             : launch_rs<int32_t, kModeBuild>(cfg, grid, a, s);
  return mode == kModeSwap ? launch_rs<float, kModeSwap>(cfg, grid, a, s)
                           : launch_rs<float, kModeBuild>(cfg, grid, a, s);
}

}  // namespace km

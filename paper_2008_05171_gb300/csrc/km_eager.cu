// km_eager.cu -- the eager SWAP variants in one persistent launch:
// FasterPAM (Alg. 4: scan the points cyclically, apply the first improving
// swap at once) and FastCLARANS (Sec. 3.4: the same over the caller's random
// draws, stopping after maxneighbor consecutive failures).
//
// Both are sequential by definition: every candidate is evaluated against
// the medoids left by the previous swap.  The GPU evaluates a window of the
// next scan positions in parallel against the current state, applies the
// first improving one, and starts the next window right after it, so the
// decisions are exactly those of the sequential scan.  Swaps come every few
// dozen positions from a random start, so per swap the cost is dominated by
// latency, not bandwidth; this kernel therefore keeps the whole loop on the
// device: a cooperative grid (every CTA resident) evaluates a window (one
// candidate row per CTA at a time, streamed with 16-byte loads), meets at a
// grid barrier, takes the decision (every CTA computes the same one from
// the window results), applies the swap to its share of the points (cache
// update + next removal loss), and meets again.  A window without a swap
// costs one barrier, a window with one costs two.
//
// The grid barrier counts arrivals on one monotonic word (release add, acquire
// polls; the e-th barrier completes at (e + 1) G arrivals), so a barrier costs
// one round trip to L2 per CTA and nothing to reset (11 % less time per swap
// than an arrival counter with a separate generation word, measured).
//
// Window length: G positions (one per CTA) after a swap, doubled up to G R
// after a window without one, so a converged scan streams at full width.
// Every barrier wait is bounded (KM_E_TIMEOUT), after which each CTA exits.
#define KM_SRC_ID 4  // names this file in bounds-check reports
#include <cstdint>

#include "km_device.cuh"
#include "km_internal.h"

namespace km {

namespace {

constexpr int kEThreads = 512;
constexpr int kEWarps = kEThreads / 32;

template <class T>
struct V4e;
template <>
struct V4e<float> {
  using type = float4;
};
template <>
struct V4e<int32_t> {
  using type = int4;
};

constexpr int kEU = 8;  // row loads (4 elements each) per thread in flight in the window loop

// Elements 4q .. 4q+3 of a matrix row, streamed (read once per window).
__device__ __forceinline__ float4 ld_row4(const float* row, int q) {
  return __ldcs(reinterpret_cast<const float4*>(row) + q);
}
__device__ __forceinline__ int4 ld_row4(const int32_t* row, int q) {
  return __ldcs(reinterpret_cast<const int4*>(row) + q);
}
__device__ __forceinline__ int4 ld_row4(const uint16_t* row, int q) {
  const uint2 u = __ldcs(reinterpret_cast<const uint2*>(row) + q);
  return make_int4((int)(u.x & 0xffffu), (int)(u.x >> 16), (int)(u.y & 0xffffu), (int)(u.y >> 16));
}

template <class V>
__device__ __forceinline__ auto comp4(const V& v, int j) -> decltype(v.x) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

constexpr int kEQ = 512;  // hit queue entries per warp
constexpr int kEM = 2;    // queue entries per lane with loads in flight

// One hit (d < d_s) of candidate c at point o: case (i) of Alg. 3 when
// d < d_n (c becomes nearest: shared term d - d_n, slot near(o) gets
// d_n - d_s), else case (ii) (slot near(o) gets d - d_s); fixed point.
template <class T>
__device__ __forceinline__ void swap_hit_e(T d, T dno, T dso, int sl, long long* acc, int k,
                                           int f, KmState* st) {
  if (!KM_INB(st, sl, k)) return;
  const long long xd = Tr<T>::fx(d, f), xs = Tr<T>::fx(dso, f);
  if (d < dno) {
    const long long xn = Tr<T>::fx(dno, f);
    atomic_add_shared64(&acc[k], xd - xn);
    atomic_add_shared64(&acc[sl], xn - xs);
  } else {
    atomic_add_shared64(&acc[sl], xd - xs);
  }
}

// top-2 entries under (distance, slot) order; slot < 0 = empty
template <class T>
__device__ __forceinline__ bool e_less(T da, int sa, T db, int sb) {
  if (sb < 0) return sa >= 0;
  if (sa < 0) return false;
  return da < db || (da == db && sa < sb);
}

template <class T>
__device__ __forceinline__ void e_push(T v, int j, int& n1, T& d1, int& n2, T& d2) {
  if (e_less(v, j, d1, n1)) {
    n2 = n1;
    d2 = d1;
    n1 = j;
    d1 = v;
  } else if (e_less(v, j, d2, n2)) {
    n2 = j;
    d2 = v;
  }
}

}  // namespace

// Dynamic shared memory: k + 1 64-bit accumulators (window phase) or k
// removal-loss partials (apply phase), the medoid of every slot, and the
// per-warp hit queues (point index, distance).
template <class E>
__global__ void __launch_bounds__(kEThreads, 1) k_eager(const EagerArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  using A = long long;
  using G = typename Tr<T>::G;
  using Vec = typename V4e<T>::type;
  extern __shared__ __align__(16) long long e_acc[];  // [k + 1], then s_med[k]
  __shared__ int s_ok;
  __shared__ int s_cnt;
  __shared__ int s_list[kEThreads];
  __shared__ long long s_key[kEWarps];
  __shared__ int s_slot[kEWarps];
  __shared__ int s_first[kEWarps];
  __shared__ long long s_cntw[kEWarps];
  __shared__ long long s_stopw;
  __shared__ G s_td[kEWarps];

  KmState* st = a.st;
  if (*(volatile int*)&st->done || *(volatile int*)&st->error) return;
  const unsigned long long wlim = wait_limit(st);
  unsigned epoch = 0;
  const int n = a.n, k = a.k, f = a.fshift;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Gn = gridDim.x;
  const bool clarans = (a.flavour == kCLARANS);
  const E* D = static_cast<const E*>(a.D);
  T* dn = static_cast<T*>(a.dn);
  T* ds = static_cast<T*>(a.ds);
  A* rem = static_cast<A*>(a.removal);
  G* td2 = static_cast<G*>(a.td2);
  int32_t* s_med = reinterpret_cast<int32_t*>(e_acc + k + 1);  // medoids by slot
  int32_t* s_qo = s_med + ((k + 3) & ~3);                       // hit queues: points
  int32_t* s_qd = s_qo + kEWarps * kEQ;                         //   and distances
  for (int i = tid; i < k; i += kEThreads) s_med[i] = __ldcg(a.med + i);

  // loop state, identical in every CTA
  long long pos = st->pos, last = st->last, wl = st->win_len;
  long long fails = st->fails, evaluated = st->evaluated;
  int rb = st->rb, swaps = st->swaps, iter = st->iter, ntrace = st->ntrace;
  double book_d = st->td_book_d;
  long long book_i = st->td_book_i;
  int done = 0, buf = 0;
  const long long wmax = (long long)Gn * a.win_rows;
  if (wl < Gn) wl = Gn;
  if (wl > wmax) wl = wmax;

  while (true) {
    const long long stop = clarans ? a.draws_len : ((last < 0) ? (long long)n : last + n);
    if (!clarans && pos >= a.max_pos) break;  // iteration cap: not converged
    long long wlen = wl;
    if (pos + wlen > stop) wlen = stop - pos;
    double* wd = a.win_delta + (size_t)buf * a.win_cap;
    int32_t* wsl = a.win_slot + (size_t)buf * a.win_cap;
    // CTA 0 clears the buffers the apply phase of this window would fill
    if (blockIdx.x == 0) {
      A* rn = rem + (size_t)(rb ^ 1) * a.k_pad;
      for (int i = tid; i < k; i += kEThreads) rn[i] = 0;
      if (tid == 0) td2[rb ^ 1] = G(0);
    }
    const A* rcur = rem + (size_t)rb * a.k_pad;

    // ------------------------------------------------ window evaluation
    for (long long w = blockIdx.x; w < wlen; w += Gn) {
      const long long p = pos + w;
      const int row = clarans ? a.draws[p] : (int)(p % n);
      const bool valid = row >= 0 && row < n && !__ldcg(a.is_med + row);
      if (!valid) {
        if (tid == 0) wsl[w] = -1;
        continue;
      }
      for (int i = tid; i <= k; i += kEThreads) e_acc[i] = 0;
      __syncthreads();
      const E* rowp = D + (size_t)row * a.ld;
      const Vec* s4 = reinterpret_cast<const Vec*>(ds);
      const int n4 = (n + 3) >> 2;
      // U float4 of the row and of d_s in flight per thread before any is
      // used.  Elements with d < d_s (hits, a few per cent) go to a
      // per-warp queue in shared memory; the warp then drains it with the
      // cache loads of several entries per lane in flight before their
      // atomic updates, instead of one L2 round trip per hit and thread.
      int32_t* qo = s_qo + warp * kEQ;
      T* qd = reinterpret_cast<T*>(s_qd) + warp * kEQ;
      // (the loop bound is uniform over the CTA: every lane of a warp takes
      // part in the warp-wide scan and shuffles below)
      for (int qb = 0; qb < n4; qb += kEU * kEThreads) {
        const int q0 = qb + tid;
        Vec d4[kEU], e4[kEU];
#pragma unroll
        for (int u = 0; u < kEU; ++u) {
          const int q = q0 + u * kEThreads;
          if (q < n4) {
            d4[u] = ld_row4(rowp, q);
            e4[u] = __ldcg(s4 + q);
          }
        }
        unsigned hm = 0;  // bit 4u + j: element j of float4 u is a hit
#pragma unroll
        for (int u = 0; u < kEU; ++u) {
          const int q = q0 + u * kEThreads;
          if (q < n4) {  // padding holds -inf / INT_MIN: never a hit
#pragma unroll
            for (int j = 0; j < 4; ++j)
              hm |= (comp4(d4[u], j) < comp4(e4[u], j) ? 1u : 0u) << (4 * u + j);
          }
        }
        const int cnt = __popc(hm);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) continue;
        if (total <= kEQ) {
          int at = incl - cnt;
#pragma unroll
          for (int u = 0; u < kEU; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (hm & (1u << (4 * u + j))) {
                qo[at] = 4 * (q0 + u * kEThreads) + j;
                qd[at] = comp4(d4[u], j);
                ++at;
              }
          __syncwarp();
          for (int e0 = 0; e0 < total; e0 += 32 * kEM) {
            int oo[kEM], sl[kEM];
            T dd[kEM], dnn[kEM], dss[kEM];
#pragma unroll
            for (int m = 0; m < kEM; ++m) {
              const int e = e0 + lane + 32 * m;
              if (e < total) {
                oo[m] = qo[e];
                dd[m] = qd[e];
                dnn[m] = __ldcg(dn + oo[m]);
                dss[m] = __ldcg(ds + oo[m]);
                sl[m] = __ldcg(a.near + oo[m]);
              }
            }
#pragma unroll
            for (int m = 0; m < kEM; ++m)
              if (e0 + lane + 32 * m < total)
                swap_hit_e<T>(dd[m], dnn[m], dss[m], sl[m], e_acc, k, f, st);
          }
          __syncwarp();
        } else {
          // dense (far from converged): every lane its own hits
#pragma unroll
          for (int u = 0; u < kEU; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (hm & (1u << (4 * u + j))) {
                const int o = 4 * (q0 + u * kEThreads) + j;
                swap_hit_e<T>(comp4(d4[u], j), __ldcg(dn + o), comp4(e4[u], j),
                              __ldcg(a.near + o), e_acc, k, f, st);
              }
        }
      }
      __syncthreads();
      // best slot: least removal loss + correction, lowest slot on ties
      A bv = LLONG_MAX;
      int bs = INT_MAX;
      for (int i = tid; i < k; i += kEThreads) {
        const A v = __ldcg(rcur + i) + e_acc[i];
        if (v < bv) {
          bv = v;
          bs = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const A v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int s2 = __shfl_xor_sync(0xffffffffu, bs, o);
        if (v2 < bv || (v2 == bv && s2 < bs)) {
          bv = v2;
          bs = s2;
        }
      }
      if (lane == 0) {
        s_key[warp] = bv;
        s_slot[warp] = bs;
      }
      __syncthreads();
      if (tid == 0) {
        A b = s_key[0];
        int sl = s_slot[0];
        for (int q = 1; q < kEWarps; ++q)
          if (s_key[q] < b || (s_key[q] == b && s_slot[q] < sl)) {
            b = s_key[q];
            sl = s_slot[q];
          }
        wd[w] = Tr<T>::unfx(b + e_acc[k], f);
        wsl[w] = sl;
      }
      __syncthreads();
    }
    if (!grid_barrier(a.bar, epoch, st, &s_ok, wlim)) return;

    // ------------------------------------------------------- decision
    // first improving position of the window (all CTAs, same result)
    int fw = INT_MAX;
    for (long long w = tid; w < wlen; w += kEThreads)
      if (__ldcg(wsl + w) >= 0 && __ldcg(wd + w) < -a.tol) {
        fw = (int)w;
        break;  // positions of one thread ascend
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fw = min(fw, __shfl_xor_sync(0xffffffffu, fw, o));
    if (lane == 0) s_first[warp] = fw;
    __syncthreads();
    fw = INT_MAX;
    for (int q = 0; q < kEWarps; ++q) fw = min(fw, s_first[q]);
    __syncthreads();
    bool swap_now = false;
    int i_s = -1, c_s = -1;
    double dlt = 0.0;
    // evaluated positions (draws) before the first improving one
    long long F = 0;
    {
      long long cnt = 0;
      for (long long w = tid; w < wlen && w < fw; w += kEThreads)
        if (__ldcg(wsl + w) >= 0) ++cnt;
      cnt = warp_sum(cnt);
      if (lane == 0) s_cntw[warp] = cnt;
      __syncthreads();
      for (int q = 0; q < kEWarps; ++q) F += s_cntw[q];
      __syncthreads();
    }
    if (clarans) {
      if (fails + F >= a.maxneighbor) {
        // stop at the draw that makes the failure count reach maxneighbor:
        // the need-th evaluated draw of the window (segments per thread,
        // block scan of their counts, one thread walks its segment)
        const long long need = a.maxneighbor - fails;
        const long long L = (wlen + kEThreads - 1) / kEThreads;
        const long long w0 = (long long)tid * L, w1 = min(w0 + L, wlen);
        long long c = 0;
        for (long long w = w0; w < w1; ++w)
          if (__ldcg(wsl + w) >= 0) ++c;
        long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        if (lane == 31) s_cntw[warp] = incl;
        __syncthreads();
        long long before = incl - c;
        for (int q = 0; q < warp; ++q) before += s_cntw[q];
        if (tid == 0) s_stopw = wlen - 1;
        __syncthreads();
        if (c > 0 && before < need && need <= before + c) {
          long long seen = before;
          for (long long w = w0; w < w1; ++w)
            if (__ldcg(wsl + w) >= 0 && ++seen == need) {
              s_stopw = w;
              break;
            }
        }
        __syncthreads();
        done = 1;
        fails = a.maxneighbor;
        evaluated += need;
        pos = pos + s_stopw + 1;
      } else if (fw != INT_MAX) {
        swap_now = true;
        fails = 0;
        evaluated += F + 1;
        last = pos + fw;
        c_s = a.draws[pos + fw];
        pos = pos + fw + 1;
      } else {
        fails += F;
        evaluated += F;
        pos += wlen;
        if (pos >= stop) done = 1;
      }
    } else {
      if (fw != INT_MAX) {
        swap_now = true;
        evaluated += F + 1;
        last = pos + fw;
        c_s = (int)((pos + fw) % n);
        pos = pos + fw + 1;
      } else {
        evaluated += F;
        pos += wlen;
        if (pos >= stop) done = 1;
      }
    }
    iter += 1;
    if (swap_now) {
      i_s = __ldcg(wsl + fw);
      dlt = __ldcg(wd + fw);
      wl = Gn;
    } else {
      wl = (2 * wl < wmax) ? 2 * wl : wmax;
    }
    buf ^= 1;
    if (!swap_now) {
      if (done) break;
      continue;
    }

    // ------------------------------------------------------ apply swap
    // cache update of this CTA's points (Alg. 3 "swap roles": c_s takes
    // slot i_s), next removal loss and exact TD
    A* sacc = e_acc;
    for (int i = tid; i < k; i += kEThreads) sacc[i] = 0;
    if (tid == 0) {
      s_cnt = 0;
      s_med[i_s] = c_s;
    }
    __syncthreads();
    A* rn = rem + (size_t)(rb ^ 1) * a.k_pad;
    G tdl = G(0);
    const E* rowc = D + (size_t)c_s * a.ld;
    // a contiguous share of the points per CTA (every CTA takes part)
    const int per = (n + Gn - 1) / Gn;
    const int lo = blockIdx.x * per, hi = min(lo + per, n);
    for (int base = lo; base < hi; base += kEThreads) {
      const int o = base + tid;
      if (o < hi) {
        const T dc = (T)rowc[o];  // issued with the cache loads (used unless rescanned)
        int n1 = __ldcg(a.near + o), n2 = __ldcg(a.sec + o);
        T d1 = __ldcg(dn + o), d2 = __ldcg(ds + o);
        if (n1 == i_s || n2 == i_s) {
          s_list[atomicAdd(&s_cnt, 1)] = o;
        } else {
          if (dc < d1 || (dc == d1 && i_s < n1)) {
            n2 = n1;
            d2 = d1;
            n1 = i_s;
            d1 = dc;
          } else if (dc < d2 || (dc == d2 && i_s < n2)) {
            n2 = i_s;
            d2 = dc;
          }
          a.near[o] = n1;
          a.sec[o] = n2;
          dn[o] = d1;
          ds[o] = d2;
          if (KM_INB(st, n1, k)) atomic_add_shared64(&sacc[n1], Tr<T>::fx(d2, f) - Tr<T>::fx(d1, f));
          tdl += G(d1);
        }
      }
      __syncthreads();
      // rescans: a warp per point, lanes over the slots
      const int cnt = s_cnt;
      for (int e = warp; e < cnt; e += kEWarps) {
        const int oo = s_list[e];
        int n1 = -1, n2 = -1;
        T d1 = Tr<T>::high(), d2 = Tr<T>::high();
#pragma unroll 4
        for (int j = lane; j < k; j += 32)
          if (KM_INB(st, s_med[j], n)) e_push((T)D[(size_t)s_med[j] * a.ld + oo], j, n1, d1, n2, d2);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const int m1 = __shfl_xor_sync(0xffffffffu, n1, off);
          const int m2 = __shfl_xor_sync(0xffffffffu, n2, off);
          const T e1 = __shfl_xor_sync(0xffffffffu, d1, off);
          const T e2 = __shfl_xor_sync(0xffffffffu, d2, off);
          e_push(e1, m1, n1, d1, n2, d2);
          e_push(e2, m2, n1, d1, n2, d2);
        }
        if (lane == 0) {
          a.near[oo] = n1;
          a.sec[oo] = n2;
          dn[oo] = d1;
          ds[oo] = d2;
          if (KM_INB(st, n1, k)) atomic_add_shared64(&sacc[n1], Tr<T>::fx(d2, f) - Tr<T>::fx(d1, f));
          tdl += G(d1);
        }
      }
      __syncthreads();
      if (tid == 0) s_cnt = 0;
      __syncthreads();
    }
    tdl = warp_sum(tdl);
    if (lane == 0) s_td[warp] = tdl;
    __syncthreads();
    if (tid == 0) {
      G t = G(0);
      for (int q = 0; q < kEWarps; ++q) t += s_td[q];
      atomic_add_acc(td2 + (rb ^ 1), t);
    }
    for (int i = tid; i < k; i += kEThreads)
      if (sacc[i] != 0) atomic_add_acc(&rn[i], sacc[i]);
    if (blockIdx.x == 0 && tid == 0) {
      // medoid bookkeeping: nobody reads med[i_s] or is_med before the
      // barrier below (rescans use c_s for slot i_s)
      const int old = __ldcg(a.med + i_s);
      a.med[i_s] = c_s;
      if (KM_INB(st, old, n)) a.is_med[old] = 0;
      a.is_med[c_s] = 1;
      if (ntrace < a.trace_cap) {
        TraceRec* tr = static_cast<TraceRec*>(a.trace) + ntrace;
        tr->d = dlt;
        tr->di = (long long)dlt;
        tr->slot = i_s;
        tr->cand = c_s;
        tr->t_ns = (long long)globaltimer();
      }
    }
    ntrace += 1;
    swaps += 1;
    book_d += dlt;
    book_i += (long long)dlt;
    rb ^= 1;
    if (!grid_barrier(a.bar, epoch, st, &s_ok, wlim)) return;
  }

  if (blockIdx.x == 0 && tid == 0) {
    st->pos = pos;
    st->last = last;
    st->win_len = wl;
    st->fails = fails;
    st->evaluated = evaluated;
    st->rb = rb;
    st->swaps = swaps;
    st->iter = iter;
    st->ntrace = ntrace;
    st->td_book_d = book_d;
    st->td_book_i = book_i;
    st->accept = 0;
    st->done = done;
  }
}

// ------------------------------------------------------------- launcher
size_t eager_smem(int k) {
  return 8 * ((size_t)k + 1) + 4 * (((size_t)k + 3) & ~(size_t)3) + 8 * (size_t)kEWarps * kEQ;
}

int eager_grid(int dtype, int k) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const size_t smem = eager_smem(k);
  cudaError_t e;
  if (dtype == 0) {
    e = cudaFuncSetAttribute(k_eager<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eager<int32_t>, kEThreads, smem);
  } else if (dtype == 2) {
    e = cudaFuncSetAttribute(k_eager<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eager<uint16_t>, kEThreads, smem);
  } else {
    e = cudaFuncSetAttribute(k_eager<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eager<float>, kEThreads, smem);
  }
  if (e != cudaSuccess || per < 1) return 0;
  if (per > 2) per = 2;
  return sms * per;
}

cudaError_t launch_eager(int dtype, int grid, const EagerArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<EagerArgs*>(&a)};
  const size_t smem = eager_smem(a.k);
  if (dtype == 0)
    return cudaLaunchCooperativeKernel((const void*)k_eager<int32_t>, dim3(grid), dim3(kEThreads),
                                       args, smem, s);
  if (dtype == 2)
    return cudaLaunchCooperativeKernel((const void*)k_eager<uint16_t>, dim3(grid),
                                       dim3(kEThreads), args, smem, s);
  return cudaLaunchCooperativeKernel((const void*)k_eager<float>, dim3(grid), dim3(kEThreads),
                                     args, smem, s);
}

}  // namespace km

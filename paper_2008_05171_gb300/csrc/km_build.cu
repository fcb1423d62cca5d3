// km_build.cu -- PAM BUILD (Alg. 1) with the gains of all candidates kept
// up to date incrementally instead of re-streaming the matrix every step.
//
// Step t adds the non-medoid c with the least gain
//     g(c) = sum_o min(d(o,c) - d_n(o), 0),
// d_n(o) the distance from o to its nearest chosen medoid (step 0: the
// distance sum of c, Eq. (3)).  Adding the medoid m lowers d_n(o) only for
// the points U = {o : d(o,m) < d_n(o)}, and g(c) depends on d_n only through
// the term of each point o.  So after the commit of m every gain is brought
// to the new d_n by adding, over o in U only,
//     delta(o,c) = min(x(d(o,c)) - x(d_n'(o)), 0) - min(x(d(o,c)) - x(d_n(o)), 0)
// (x = the fixed-point value; d_n' the new, d_n the old distance), which is
// d_n - d_n' when d(o,c) < d_n', d_n - d(o,c) when d_n' <= d(o,c) < d_n, and
// 0 otherwise.  By symmetry d(o,c) = D[o*ld + c]: the update streams the
// rows of the points in U, contiguous over the candidates.  A step reads |U|
// rows instead of n - t; over a whole BUILD on clustered data the rows read
// add up to a few passes over the matrix instead of k passes.
//
// Every gain is an exact 64-bit fixed-point sum, floor(d * 2^f) per term for
// float data (f from the matrix scan, so that n * max|d| * 2^f < 2^60), the
// integer itself for integer data; additions in any order give the same
// bits, so the per-candidate atomics are deterministic and the greedy choice
// (least gain, lowest index on ties) is that of the plain pass evaluated in
// the same arithmetic.
//
// Kernels, one launch each per step, no waits between CTAs:
//   k_build_update   CTA (tile, group): 1024 candidate columns x its share of
//                    the listed rows; each thread owns 4 consecutive
//                    candidates and keeps their deltas in registers, then
//                    adds them to the gains with 64-bit integer atomics.  The
//                    last CTA of a column tile (ticket) takes the tile's best
//                    non-medoid; the last tile takes the grid's best and
//                    writes the step's choice to the device state.
//   k_build_add      commits the chosen medoid: d_n, the exact TD, the
//                    medoid arrays and the list U of the points whose d_n
//                    dropped (warp-aggregated appends).
#define KM_SRC_ID 3  // names this file in bounds-check reports
#include <type_traits>

#include "km_device.cuh"
#include "km_internal.h"

namespace km {

constexpr int kBuThreads = 256;              // 4 candidate columns each
constexpr int kBuCols = 4 * kBuThreads;      // columns per tile (= kChunk)
constexpr int kBuMinRows = 8;                // listed rows per CTA, at least
constexpr int kBuUnroll = 8;                 // row loads in flight per thread
static_assert(kBuCols == kChunk, "a tile spans one padding unit of n");

struct BuildRowEntry {  // one listed point, staged in shared memory
  long long xn, xo;     // fixed-point new / old d_n
  int o;                // point index (its row of D)
  uint32_t vn, vo;      // new / old d_n as stored (raw bits)
  int pad;
};

template <class T>
__device__ __forceinline__ T bu_high();
template <>
__device__ __forceinline__ float bu_high<float>() {
  return __int_as_float(0x7f800000);
}
template <>
__device__ __forceinline__ int32_t bu_high<int32_t>() {
  return INT_MAX;
}

// Raw 32-bit storage of a value (the list keeps float and int32 alike).
__device__ __forceinline__ uint32_t bu_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t bu_bits(int32_t v) { return (uint32_t)v; }
template <class T>
__device__ __forceinline__ T bu_from(uint32_t b);
template <>
__device__ __forceinline__ float bu_from<float>(uint32_t b) {
  return __uint_as_float(b);
}
template <>
__device__ __forceinline__ int32_t bu_from<int32_t>(uint32_t b) {
  return (int32_t)b;
}

__device__ __forceinline__ float comp(const float4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
__device__ __forceinline__ int32_t comp(const int4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// The contribution of one listed row to four consecutive candidates:
//   distance sums (step 0):       x(d)
//   first gains (after step 0):   min(x(d) - x(d_n'), 0)
//   later steps:                  the change of min(x(d) - x(d_n), 0) as d_n
//                                 drops to d_n' (see the file comment).
// The value comparisons decide the same cases as the fixed-point ones
// (x is monotone, and a case that only the rounding merges contributes 0).
template <class T, int MODE, class Vec>
__device__ __forceinline__ void bu_accumulate(long long (&acc)[4], const Vec& d,
                                              const BuildRowEntry& e, int f) {
  const T vn = bu_from<T>(e.vn), vo = bu_from<T>(e.vo);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T v = comp(d, j);
    if (MODE == kBuildColsum) {
      acc[j] += Tr<T>::fx(v, f);
    } else if (MODE == kBuildFirst) {
      if (v < vn) acc[j] += Tr<T>::fx(v, f) - e.xn;
    } else if (v < vo) {
      acc[j] += (v < vn) ? (e.xo - e.xn) : (e.xo - Tr<T>::fx(v, f));
    }
  }
}

// ------------------------------------------------------------ update pass
template <class E, int MODE>
__global__ void __launch_bounds__(kBuThreads) k_build_update(const BuildArgs a) {
  using T = typename Val<E>::type;
  using Vec = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
  __shared__ BuildRowEntry rows[kBuThreads];
  __shared__ Key<long long> wk[kBuThreads / 32];
  __shared__ int s_last;

  KmState* st = a.st;
  if (st->error) return;  // uniform for the whole launch
  BuildAux* aux = a.aux;
  Key<long long>* partials = static_cast<Key<long long>*>(a.partials);
  const int n = a.n, f = a.fshift;
  const int tile = blockIdx.x, grp = blockIdx.y, groups = gridDim.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int col = tile * kBuCols + 4 * tid;

  // rows of this CTA: a contiguous share of the list (or of 0..n-1), at
  // least kBuMinRows of them unless the list is shorter.  The groups past
  // the list's share leave at once and take no ticket; the count they read
  // stays unchanged during the launch (the next commit appends to the other
  // counter, which this launch clears first).
  long long cnt =
      (MODE == kBuildColsum) ? (long long)n : (long long)__ldcg(&aux->cnt[a.cur]);
  if (!KM_INB(st, cnt, (long long)n + 1)) cnt = 0;  // the list holds at most n points
  long long g_eff = (cnt + kBuMinRows - 1) / kBuMinRows;
  if (g_eff > groups) g_eff = groups;
  if (g_eff < 1) g_eff = 1;
  if (grp >= g_eff) return;  // uniform for the CTA
  if (tile == 0 && grp == 0 && tid == 0) aux->cnt[a.cur ^ 1] = 0u;
  const long long r0 = cnt * grp / g_eff;
  const long long r1 = cnt * (grp + 1) / g_eff;

  long long acc[4] = {0, 0, 0, 0};
  const E* D = static_cast<const E*>(a.D);
  const bool cvalid = col < n;  // col and ld are multiples of 4: the vector is in the row
  for (long long b = r0; b < r1; b += kBuThreads) {
    const int m = (int)((r1 - b < kBuThreads) ? (r1 - b) : kBuThreads);
    __syncthreads();  // the previous batch is consumed
    if (tid < m) {
      BuildRowEntry e;
      const long long i = b + tid;
      e.pad = 0;
      if (MODE == kBuildColsum) {
        e.o = (int)i;
        e.vn = 0u;
        e.vo = 0u;
        e.xn = 0;
        e.xo = 0;
      } else {
        e.o = a.list[i];
        if (!KM_INB(st, e.o, n)) e.o = 0;  // a row that exists; the error is recorded
        e.vn = a.lvn[i];
        e.vo = a.lvo[i];
        e.xn = Tr<T>::fx(bu_from<T>(e.vn), f);
        e.xo = (MODE == kBuildStep) ? Tr<T>::fx(bu_from<T>(e.vo), f) : 0;
      }
      rows[tid] = e;
    }
    __syncthreads();
    if (!cvalid) continue;
    constexpr int U = kBuUnroll;
    for (int q = 0; q < m; q += U) {
      // all loads of the group first (predicated), then the arithmetic
      Vec d[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q + u < m) d[u] = ld4e(D + (size_t)rows[q + u].o * (size_t)a.ld + col);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (q + u < m) bu_accumulate<T, MODE>(acc, d[u], rows[q + u], f);
    }
  }
  if (cvalid && r1 > r0) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (col + j < n && acc[j] != 0) atomic_add_acc(a.cgain + col + j, acc[j]);
  }

  // ---------------------------------------------- last CTA of the tile
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned t = atomicAdd(&a.tticket[tile], 1u);
    s_last = (t == (unsigned)g_eff - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  Key<long long> best;
  best.d = LLONG_MAX;
  best.slot = 0;
  best.cand = INT_MAX;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = col + j;
    if (c < n && !__ldcg(a.is_med + c)) {
      Key<long long> kk;
      kk.d = __ldcg(a.cgain + c);
      kk.slot = 0;
      kk.cand = c;
      if (key_less(kk, best)) best = kk;
    }
  }
  best = warp_min_key(best);
  if (lane == 0) wk[warp] = best;
  __syncthreads();
  if (tid == 0) {
    Key<long long> b = wk[0];
    for (int w = 1; w < kBuThreads / 32; ++w)
      if (key_less(wk[w], b)) b = wk[w];
    partials[tile] = b;
    a.tticket[tile] = 0u;  // every CTA of this tile has arrived
    __threadfence();
    const unsigned t = atomicAdd(&aux->gticket, 1u);
    s_last = (t == gridDim.x - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;

  // ------------------------------------------- last tile: the step's choice
  __threadfence();
  if (warp == 0) {
    Key<long long> b;
    b.d = LLONG_MAX;
    b.slot = 0;
    b.cand = INT_MAX;
    for (int g = lane; g < (int)gridDim.x; g += 32) {
      const Key<long long> v = ld_cg_key(partials + g);
      if (key_less(v, b)) b = v;
    }
    b = warp_min_key(b);
    if (lane == 0) {
      st->build_cand = (b.cand < n) ? b.cand : -1;
      st->build_gain_i = b.d;
      st->build_gain_d = Tr<T>::unfx(b.d, f);
      st->build_td_d = 0.0;
      st->build_td_i = 0;
      aux->rows_total += (unsigned long long)cnt;
      aux->gticket = 0u;
    }
  }
}

// --------------------------------------------------------------- commit
// Adds the chosen point c as medoid `build_step`: d_n(o) = min(d_n(o),
// d(c,o)) (step 0: d(c,o)), the exact TD of the new medoid set, the medoid
// arrays, the TD bookkeeping, and the list of the points whose d_n dropped
// with their new and old values.  Step 0 also clears the gains (they held
// the distance sums).
template <class E>
__global__ void __launch_bounds__(kBuThreads) k_build_add(const BuildArgs a) {
  using T = typename Val<E>::type;
  using G = typename Tr<T>::G;
  __shared__ G scratch[kBuThreads / 32];
  KmState* st = a.st;
  if (st->error) return;
  const int c = st->build_cand;
  if (c < 0 || c >= a.n) return;  // uniform: nothing was chosen
  const int n = a.n;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const E* D = static_cast<const E*>(a.D);
  T* bdn = static_cast<T*>(a.bdn);
  bool changed = false;
  T v = T(0), prev = bu_high<T>();
  G local = G(0);
  if (o < n) {
    v = (T)D[(size_t)c * (size_t)a.ld + o];
    T cur = v;
    if (a.first) {
      changed = true;
    } else {
      prev = bdn[o];
      if (v < prev)
        changed = true;
      else
        cur = prev;
    }
    bdn[o] = cur;
    local = G(cur);
  } else if (o < a.n_pad) {
    bdn[o] = Tr<T>::low();  // padding: never above a distance
  }
  if (a.first && o < a.n_pad) a.cgain[o] = 0;

  // warp-aggregated append to the list U
  const unsigned m = __ballot_sync(0xffffffffu, changed);
  if (m) {
    unsigned base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(&a.aux->cnt[a.cur], (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (changed) {
      unsigned lt;
      asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
      const unsigned idx = base + (unsigned)__popc(m & lt);
      if (KM_INB(a.st, idx, a.n_pad)) {
        a.list[idx] = o;
        a.lvn[idx] = bu_bits(v);
        a.lvo[idx] = bu_bits(prev);
      }
    }
  }

  // exact TD of the new medoid set
  G s = warp_sum(local);
  if (lane == 0) scratch[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    G bs = G(0);
    for (int w = 0; w < kBuThreads / 32; ++w) bs += scratch[w];
    atomic_add_acc(std::is_same<G, double>::value ? reinterpret_cast<G*>(&st->build_td_d)
                                                  : reinterpret_cast<G*>(&st->build_td_i),
                   bs);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && KM_INB(st, st->build_step, a.k)) {
    const int step = st->build_step;
    a.med[step] = c;
    a.is_med[c] = 1;
    if (a.gains) a.gains[step] = st->build_gain_d;
    if (a.first) {
      st->td_book_d = st->build_gain_d;
      st->td_book_i = st->build_gain_i;
    } else {
      st->td_book_d += st->build_gain_d;
      st->td_book_i += st->build_gain_i;
    }
    st->build_step = step + 1;
  }
}

// -------------------------------------------------------------- launchers
int build_update_groups(int n, int sms) {
  const int tiles = (n + kBuCols - 1) / kBuCols;
  // up to 8 CTAs per SM in all: a short list spreads over enough CTAs that
  // each issues its (at most kBuMinRows) row loads at once; the CTAs past
  // the list's share exit at once
  int g = (8 * sms + tiles - 1) / tiles;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return g;
}

template <class E>
static cudaError_t launch_update_t(int mode, int groups, const BuildArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.n + kBuCols - 1) / kBuCols), (unsigned)groups);
  switch (mode) {
    case kBuildColsum:
      k_build_update<E, kBuildColsum><<<grid, kBuThreads, 0, s>>>(a);
      break;
    case kBuildFirst:
      k_build_update<E, kBuildFirst><<<grid, kBuThreads, 0, s>>>(a);
      break;
    default:
      k_build_update<E, kBuildStep><<<grid, kBuThreads, 0, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_update(int dtype, int mode, int groups, const BuildArgs& a,
                                cudaStream_t s) {
  if (dtype == 0) return launch_update_t<int32_t>(mode, groups, a, s);
  if (dtype == 2) return launch_update_t<uint16_t>(mode, groups, a, s);
  return launch_update_t<float>(mode, groups, a, s);
}

cudaError_t launch_build_add(int dtype, const BuildArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(a.n_pad / kBuThreads);
  if (dtype == 0)
    k_build_add<int32_t><<<blocks, kBuThreads, 0, s>>>(a);
  else if (dtype == 2)
    k_build_add<uint16_t><<<blocks, kBuThreads, 0, s>>>(a);
  else
    k_build_add<float><<<blocks, kBuThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace km

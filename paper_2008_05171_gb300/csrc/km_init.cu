// km_init.cu -- the cheap initialisations of Sec. 3.3 on the matrix form:
// distance-weighted seeding (the k-means++ strategy of Sec. 2.3 with plain
// distances as weights) and LAB (Linear Approximative BUILD: BUILD's gain
// over a fresh random subsample before each choice).  Either start feeds
// FasterPAM, which the paper recommends over BUILD once swapping is cheap
// (Sec. 4.3, Sec. 6).
//
// Both run all k choices inside one launch of a single 1024-thread CTA: a
// choice depends on every earlier one, and its work (one matrix row of n
// entries, plus s^2 entries for LAB) is far too small to spread over the
// GPU.  The random numbers are the caller's: uniform numbers u_t for the
// weighted draws, subsample ranks for LAB.  Weights and gains are exact
// 64-bit fixed point (distances enter as floor(x 2^f), the scale of the SWAP
// sums; integer distances unchanged), so every choice is independent of the
// summation order.
#define KM_SRC_ID 7  // names this file in bounds-check reports
#include <cstdint>

#include "km_device.cuh"
#include "km_internal.h"

namespace km {

namespace {

constexpr int kInitThreads = 1024;
constexpr int kInitWarps = kInitThreads / 32;

template <class A>
__device__ __forceinline__ A warp_incl_scan(A v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const A t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive prefix sum of one value per thread; *total gets the
// sum.  Uses s_w[kInitWarps]; contains two __syncthreads.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* s_w,
                                                     long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long incl = warp_incl_scan(v, lane);
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  long long wsum = (lane < kInitWarps) ? s_w[lane] : 0;
  const long long wincl = warp_incl_scan(wsum, lane);
  const long long before = __shfl_sync(0xffffffffu, wincl - wsum, warp);
  *total = __shfl_sync(0xffffffffu, wincl, kInitWarps - 1);
  __syncthreads();
  return before + incl - v;
}

}  // namespace

// ------------------------------------------------------ distance-weighted
// Draw 0: floor(u_0 n).  Draw t >= 1: weights w_o = fx(d_n(o)), their total
// W, threshold T = floor(u_t W) in FP64 (clamped to [0, W-1]); the pick is
// the lowest o whose running weight sum exceeds T.  W = 0 (every point
// coincides with a medoid): the lowest point not drawn yet.
//
// Per draw: the row of the previous pick updates d_n (coalesced, a warp per
// 32-point chunk) and each warp stores its chunks' weight sums; a block scan
// over contiguous runs of chunk sums finds the chunk holding T, and one
// warp scans inside it.
template <class E>
__global__ void __launch_bounds__(kInitThreads) k_init_weighted(const InitArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  __shared__ long long s_w[kInitWarps];
  __shared__ long long s_rem;
  __shared__ int s_chunk;
  __shared__ int s_pick;
  const E* D = static_cast<const E*>(a.D);
  T* dn = static_cast<T*>(a.dn);
  long long* csum = a.csum;
  const int n = a.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nch = (n + 31) >> 5;  // 32-point chunks
  const int per = (nch + kInitThreads - 1) / kInitThreads;

  for (int o = tid; o < n; o += kInitThreads) a.flags[o] = 0;
  if (tid == 0) {
    long long c = (long long)floor(a.u[0] * (double)n);
    c = c > n - 1 ? n - 1 : (c < 0 ? 0 : c);
    s_pick = (int)c;
    a.med[0] = (int32_t)c;
  }
  __syncthreads();
  int pick = s_pick;
  if (tid == 0) a.flags[pick] = 1;

  for (int t = 1; t < a.k; ++t) {
    // d_n update with the previous pick's row, chunk sums of the weights
    const E* row = D + (size_t)pick * (size_t)a.ld;
    for (int q = warp; q < nch; q += kInitWarps) {
      const int o = (q << 5) + lane;
      long long w = 0;
      if (o < n) {
        const T v = row[o];
        const T cur = (t == 1) ? v : (v < dn[o] ? v : dn[o]);
        dn[o] = cur;
        w = Tr<T>::fx(cur, a.fshift);
      }
      w = warp_sum(w);
      if (lane == 0) csum[q] = w;
    }
    __syncthreads();
    // which chunk holds the threshold
    long long part = 0;
    const int q0 = tid * per, q1 = min(q0 + per, nch);
    for (int q = q0; q < q1; ++q) part += csum[q];
    long long W = 0;
    const long long before = block_excl_scan(part, s_w, &W);
    if (W > 0) {
      long long Tt = (long long)floor(a.u[t] * (double)W);
      Tt = Tt > W - 1 ? W - 1 : (Tt < 0 ? 0 : Tt);
      if (part > 0 && before <= Tt && Tt < before + part) {
        long long acc = before;
        for (int q = q0; q < q1; ++q) {
          const long long cq = csum[q];
          if (acc + cq > Tt) {
            s_chunk = q;
            s_rem = Tt - acc;
            break;
          }
          acc += cq;
        }
      }
      __syncthreads();
      if (warp == 0) {
        const int q = s_chunk;
        const int o = (q << 5) + lane;
        const long long w = (o < n) ? Tr<T>::fx(dn[o], a.fshift) : 0;
        const long long incl = warp_incl_scan(w, lane);
        const unsigned hit = __ballot_sync(0xffffffffu, incl > s_rem);
        if (lane == 0) s_pick = (q << 5) + __ffs(hit) - 1;
      }
    } else {
      // every weight is zero: the lowest point not drawn yet
      int lo = INT_MAX;
      for (int o = tid; o < n; o += kInitThreads)
        if (!a.flags[o]) {
          lo = o;
          break;
        }
      for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      if (lane == 0) s_w[warp] = lo;
      __syncthreads();
      if (warp == 0) {
        int v = (int)s_w[lane];
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) s_pick = v;
      }
    }
    __syncthreads();
    pick = s_pick;
    if (!KM_INB(a.st, pick, n)) pick = 0;  // a row that exists; the error is recorded
    if (tid == 0) {
      a.med[t] = pick;
      a.flags[pick] = 1;
    }
  }
}

// ------------------------------------------------------------------- LAB
// Step t: the subsample is given as ranks among the n - t non-medoids in
// index order (negative = unused entry); rank r maps to the point
// p = r + #{j : m_(j) - j <= r} over the sorted medoids m_(0) < m_(1) < ...
// (m_(j) - j counts the non-medoids before m_(j)).  Every subsample point c
// gets gain(c) = sum_{o in S} min(fx(d(o,c)) - fx(d_n(o)), 0), or at step 0
// sum_{o in S} fx(d(o,c)); the least (gain, point) wins.  Then d_n takes the
// row of the new medoid.  Dynamic shared memory: sorted medoids (k int32),
// subsample points (s int32), fx(d_n) of the subsample (s int64).
template <class E>
__global__ void __launch_bounds__(kInitThreads) k_init_lab(const InitArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  extern __shared__ __align__(16) unsigned char sm_raw[];
  long long* s_dn = reinterpret_cast<long long*>(sm_raw);
  int32_t* s_pts = reinterpret_cast<int32_t*>(s_dn + a.s);
  int32_t* s_sorted = s_pts + a.s;
  __shared__ long long s_g[kInitWarps];
  __shared__ int s_c[kInitWarps];
  __shared__ int s_pick;
  const E* D = static_cast<const E*>(a.D);
  T* dn = static_cast<T*>(a.dn);
  const int n = a.n, s = a.s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int t = 0; t < a.k; ++t) {
    // subsample points and their fixed-point d_n
    for (int j = tid; j < s; j += kInitThreads) {
      const int r = a.ranks[(size_t)t * s + j];
      int p = -1;
      if (r >= 0) {
        int lo = 0, hi = t;  // count of sorted medoids with m_(j) - j <= r
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_sorted[mid] - mid <= r) lo = mid + 1;
          else hi = mid;
        }
        p = r + lo;
        if (!KM_INB(a.st, p, n)) p = -1;
      }
      s_pts[j] = p;
      s_dn[j] = (p >= 0 && t > 0) ? Tr<T>::fx(dn[p], a.fshift) : 0;
    }
    __syncthreads();
    // gains: a warp per candidate, lanes over the subsample
    long long best = LLONG_MAX;
    int bc = INT_MAX;
    for (int jc = warp; jc < s; jc += kInitWarps) {
      const int c = s_pts[jc];
      if (c < 0) continue;
      const E* row = D + (size_t)c * (size_t)a.ld;
      long long g = 0;
      for (int jo = lane; jo < s; jo += 32) {
        const int o = s_pts[jo];
        if (o < 0) continue;
        const long long v = Tr<T>::fx(row[o], a.fshift);
        if (t == 0) g += v;
        else {
          const long long dlt = v - s_dn[jo];
          g += dlt < 0 ? dlt : 0;
        }
      }
      g = warp_sum(g);
      if (g < best || (g == best && c < bc)) {
        best = g;
        bc = c;
      }
    }
    if (lane == 0) {
      s_g[warp] = best;
      s_c[warp] = bc;
    }
    __syncthreads();
    if (warp == 0) {
      long long g = s_g[lane];
      int c = s_c[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long g2 = __shfl_xor_sync(0xffffffffu, g, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, c, o);
        if (g2 < g || (g2 == g && c2 < c)) {
          g = g2;
          c = c2;
        }
      }
      if (lane == 0) {
        s_pick = c;
        a.med[t] = c;
        if (a.gains) a.gains[t] = Tr<T>::unfx(g, a.fshift);
        // insert into the sorted medoid list
        int j = t;
        while (j > 0 && s_sorted[j - 1] > c) {
          s_sorted[j] = s_sorted[j - 1];
          --j;
        }
        s_sorted[j] = c;
      }
    }
    __syncthreads();
    const int pick = s_pick;
    if (pick < 0 || pick >= n) {  // an empty subsample (the host rejects it)
      if (tid == 0) a.st->error = 1;
      return;
    }
    if (t + 1 < a.k) {
      const E* row = D + (size_t)pick * (size_t)a.ld;
      for (int o = tid; o < n; o += kInitThreads) {
        const T v = row[o];
        dn[o] = (t == 0 || v < dn[o]) ? v : dn[o];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- launchers
size_t init_lab_smem(int k, int s) { return (size_t)s * 12 + (size_t)k * 4; }

cudaError_t launch_init_weighted(int dtype, const InitArgs& a, cudaStream_t st) {
  if (dtype == 0)
    k_init_weighted<int32_t><<<1, kInitThreads, 0, st>>>(a);
  else if (dtype == 2)
    k_init_weighted<uint16_t><<<1, kInitThreads, 0, st>>>(a);
  else
    k_init_weighted<float><<<1, kInitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init_lab(int dtype, const InitArgs& a, cudaStream_t st) {
  const size_t smem = init_lab_smem(a.k, a.s);
  cudaError_t e;
  if (dtype == 0) {
    e = cudaFuncSetAttribute(k_init_lab<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_init_lab<int32_t><<<1, kInitThreads, smem, st>>>(a);
  } else if (dtype == 2) {
    e = cudaFuncSetAttribute(k_init_lab<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_init_lab<uint16_t><<<1, kInitThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_init_lab<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_init_lab<float><<<1, kInitThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace km

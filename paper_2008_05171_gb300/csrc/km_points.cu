// km_points.cu -- per-point kernels of the SWAP and BUILD loops:
//
//   k_cache_init      nearest / second-nearest slot and distance of every
//                     point (Sec. 2), the removal loss Delta^{-m_i} (Eq. (7))
//                     and the exact TD (Eq. (2)) for the current medoids.
//   k_apply           performs the pending swap (Alg. 3 "swap roles"): the
//                     new medoid takes the slot of the removed one; the cache
//                     is updated incrementally (points whose nearest or
//                     second nearest was the removed slot are rescanned over
//                     all k medoids by a whole warp), and the removal loss /
//                     TD of the next pass are accumulated on the way.
//   k_build_commit    adds the chosen BUILD medoid and updates d_n (Alg. 1).
//   k_fp2_try         FastPAM2: exact Delta of one queued per-slot swap
//                     against the current cache, by Eq. (5).
//   k_matrix_scan     largest entry (fixed-point scale) and invalid values.
//   k_matrix_check    optional input check: zero diagonal, symmetry.
//
// One thread per point; d(x_o, x_m) is read as D[m*ld + o] so a warp reads
// 32 consecutive elements of a medoid row.  The template parameter is the
// stored element type (float, int32, or uint16 widened to int32).
// Grid-wide results use a last-block-done ticket in the device state.
#define KM_SRC_ID 2  // names this file in bounds-check reports
#include <type_traits>

#include "km_device.cuh"
#include "km_internal.h"

namespace km {

constexpr int kPtThreads = 256;

// bitwise inequality, zero test and value test of the input check
__device__ __forceinline__ bool memcmp_bits(float a, float b) {
  return __float_as_uint(a) != __float_as_uint(b);
}
__device__ __forceinline__ bool memcmp_bits(int32_t a, int32_t b) { return a != b; }
__device__ __forceinline__ bool memcmp_bits(uint16_t a, uint16_t b) { return a != b; }
__device__ __forceinline__ bool is_zero(float a) { return a == 0.f; }
__device__ __forceinline__ bool is_zero(int32_t a) { return a == 0; }
__device__ __forceinline__ bool is_zero(uint16_t a) { return a == 0; }
__device__ __forceinline__ bool bad_value(float a) { return !(a >= 0.f) || isinf(a); }
__device__ __forceinline__ bool bad_value(int32_t a) { return a < 0; }
__device__ __forceinline__ bool bad_value(uint16_t) { return false; }

template <class A>
__device__ __forceinline__ A block_sum(A v, A* scratch) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) scratch[w] = v;
  __syncthreads();
  A r = A(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += scratch[i];
  __syncthreads();
  return r;  // valid in thread 0
}

// top-2 insertion under the lexicographic (distance, slot) order, with
// slots offered in ascending order (strict comparisons keep the lowest slot)
template <class T>
__device__ __forceinline__ void top2_push(T v, int j, int& n1, T& d1, int& n2, T& d2) {
  if (n1 < 0 || v < d1) {
    n2 = n1;
    d2 = d1;
    n1 = j;
    d1 = v;
  } else if (n2 < 0 || v < d2) {
    n2 = j;
    d2 = v;
  }
}

// ------------------------------------------------------------ cache init
template <class E>
__global__ void __launch_bounds__(kPtThreads) k_cache_init(const PointArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  using A = typename Tr<T>::A;  // removal loss (fixed point / int64)
  using G = typename Tr<T>::G;  // TD
  extern __shared__ __align__(16) unsigned char sm[];
  A* sacc = reinterpret_cast<A*>(sm);
  G* scratch = reinterpret_cast<G*>(sacc + a.k);
  __shared__ int is_last;
  KmState* st = a.st;
  const int k = a.k, n = a.n, f = a.fshift;
  const int rb = st->rb;
  for (int i = threadIdx.x; i < k; i += blockDim.x) sacc[i] = A(0);
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const E* D = static_cast<const E*>(a.D);
  T* dn = static_cast<T*>(a.dn);
  T* ds = static_cast<T*>(a.ds);
  G tdl = G(0);
  if (o < n) {
    int n1 = -1, n2 = -1;
    T d1 = Tr<T>::high(), d2 = Tr<T>::high();
    for (int j = 0; j < k; ++j) {
      const int m = a.med[j];
      if (!KM_INB(st, m, a.m)) continue;
      const T v = D[(size_t)m * a.ld + o];
      top2_push(v, j, n1, d1, n2, d2);
    }
    a.near[o] = n1;
    a.sec[o] = n2;
    dn[o] = d1;
    ds[o] = (n2 < 0) ? Tr<T>::high() : d2;
    if (n2 >= 0) atomic_add_shared64(&sacc[n1], Tr<T>::fx(d2, f) - Tr<T>::fx(d1, f));
    tdl = G(d1);
  } else if (o < a.n_pad) {
    a.near[o] = 0;
    a.sec[o] = 0;
    dn[o] = Tr<T>::low();  // sentinels: d < low never holds
    ds[o] = Tr<T>::low();
  }
  const G bs = block_sum(tdl, scratch);
  A* rem = static_cast<A*>(a.removal) + (size_t)rb * a.k_pad;
  if (threadIdx.x == 0) atomic_add_acc(static_cast<G*>(a.td2) + rb, bs);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (sacc[i] != A(0)) atomic_add_acc(&rem[i], sacc[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    const G td0 = static_cast<volatile G*>(a.td2)[rb];
    st->td_book_d = to_double(td0);
    st->td_book_i = (long long)td0;
    st->ticket = 0;
  }
}

// -------------------------------------------------------------- apply swap
// Lexicographic (distance, slot) order of cache entries; slot < 0 = empty.
template <class T>
__device__ __forceinline__ bool entry_less(T da, int sa, T db, int sb) {
  if (sb < 0) return sa >= 0;
  if (sa < 0) return false;
  return da < db || (da == db && sa < sb);
}

// Merge of two top-2 lists: the two least entries of {a1, a2, b1, b2}.
template <class T>
__device__ __forceinline__ void top2_merge(int& n1, T& d1, int& n2, T& d2, int m1, T e1, int m2,
                                           T e2) {
  if (entry_less(e1, m1, d1, n1)) {
    // e1 is the least; the second is the lesser of d1 and e2
    if (entry_less(e2, m2, d1, n1)) {
      n2 = m2;
      d2 = e2;
    } else {
      n2 = n1;
      d2 = d1;
    }
    n1 = m1;
    d1 = e1;
  } else if (entry_less(e1, m1, d2, n2)) {
    n2 = m1;
    d2 = e1;
  }
}

template <class E>
__global__ void __launch_bounds__(kPtThreads) k_apply(const PointArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  using A = typename Tr<T>::A;  // removal loss (fixed point / int64)
  using G = typename Tr<T>::G;  // TD
  extern __shared__ __align__(16) unsigned char sm[];
  A* sacc = reinterpret_cast<A*>(sm);
  G* scratch = reinterpret_cast<G*>(sacc + a.k);
  const int f = a.fshift;
  __shared__ int is_last;
  __shared__ int s_cnt;
  __shared__ int s_list[kPtThreads];
  KmState* st = a.st;
  if (st->error || !st->accept) return;  // uniform for the launch
  const int k = a.k, n = a.n;
  const int i_s = st->best_slot, c_s = st->best_cand;
  if (!KM_INB(st, i_s, k) || !KM_INB(st, c_s, a.m)) return;  // uniform for the launch
  const int rb = st->rb;
  for (int i = threadIdx.x; i < k; i += blockDim.x) sacc[i] = A(0);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const E* D = static_cast<const E*>(a.D);
  T* dn = static_cast<T*>(a.dn);
  T* ds = static_cast<T*>(a.ds);
  G tdl = G(0);
  if (o < n && KM_INB(st, a.near[o], k)) {
    int n1 = a.near[o], n2 = a.sec[o];
    T d1 = dn[o], d2 = ds[o];
    if (n1 == i_s || n2 == i_s) {
      // the removed medoid was nearest or second: a full rescan, done below
      // by a whole warp
      s_list[atomicAdd(&s_cnt, 1)] = threadIdx.x;
    } else {
      // only the new medoid enters: top-2 of {nearest, second, new}
      const T dc = D[(size_t)c_s * a.ld + o];
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
      atomic_add_shared64(&sacc[n1], Tr<T>::fx(d2, f) - Tr<T>::fx(d1, f));
      tdl = G(d1);
    }
  }
  __syncthreads();
  // Rescans: a warp per point, lanes over the slots (each lane keeps the
  // top-2 of its slots, then a butterfly merge under (distance, slot)).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = s_cnt;
  for (int e = warp; e < cnt; e += kPtThreads / 32) {
    const int oo = blockIdx.x * blockDim.x + s_list[e];
    int n1 = -1, n2 = -1;
    T d1 = Tr<T>::high(), d2 = Tr<T>::high();
    for (int j = lane; j < k; j += 32) {
      const int m = (j == i_s) ? c_s : a.med[j];
      if (!KM_INB(st, m, a.m)) continue;
      top2_push((T)D[(size_t)m * a.ld + oo], j, n1, d1, n2, d2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int m1 = __shfl_xor_sync(0xffffffffu, n1, off);
      const int m2 = __shfl_xor_sync(0xffffffffu, n2, off);
      const T e1 = __shfl_xor_sync(0xffffffffu, d1, off);
      const T e2 = __shfl_xor_sync(0xffffffffu, d2, off);
      top2_merge(n1, d1, n2, d2, m1, e1, m2, e2);
    }
    if (lane == 0 && n1 >= 0) {
      a.near[oo] = n1;
      a.sec[oo] = n2;
      dn[oo] = d1;
      ds[oo] = d2;
      atomic_add_shared64(&sacc[n1], Tr<T>::fx(d2, f) - Tr<T>::fx(d1, f));
      tdl += G(d1);
    }
  }
  const G bs = block_sum(tdl, scratch);
  A* rem = static_cast<A*>(a.removal) + (size_t)(rb ^ 1) * a.k_pad;
  if (threadIdx.x == 0) atomic_add_acc(static_cast<G*>(a.td2) + (rb ^ 1), bs);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (sacc[i] != A(0)) atomic_add_acc(&rem[i], sacc[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    const int old = a.med[i_s];
    a.med[i_s] = c_s;
    if (KM_INB(st, old, a.m)) a.is_med[old] = 0;
    a.is_med[c_s] = 1;
    const int nt = st->ntrace;
    if (nt < a.trace_cap) {
      TraceRec* tr = static_cast<TraceRec*>(a.trace) + nt;
      tr->d = st->best_d;
      tr->di = st->best_i;
      tr->slot = i_s;
      tr->cand = c_s;
      tr->t_ns = (long long)globaltimer();
    }
    st->ntrace = nt + 1;
    st->swaps += 1;
    st->td_book_d += st->best_d;
    st->td_book_i += st->best_i;
    st->accept = 0;
    st->rb = rb ^ 1;
    st->ticket = 0;
  }
}

// ------------------------------------------------------------ BUILD commit
template <class E>
__global__ void __launch_bounds__(kPtThreads) k_build_commit(const PointArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  using A = typename Tr<T>::G;
  __shared__ A scratch[kPtThreads / 32];
  KmState* st = a.st;
  if (st->error) return;
  const int n = a.n;
  const int c = st->build_cand;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const E* D = static_cast<const E*>(a.D);
  T* bdn = static_cast<T*>(a.bdn);
  A local = A(0);
  if (c >= 0 && c < a.m) {
    if (o < n) {
      const T v = D[(size_t)c * a.ld + o];
      T cur = v;
      if (!a.build_first) {
        const T prev = bdn[o];
        if (!(v < prev)) cur = prev;
      }
      bdn[o] = cur;
      local = A(cur);
    } else if (o < a.n_pad) {
      bdn[o] = Tr<T>::low();  // padding: never above a distance
    }
  }
  const A bs = block_sum(local, scratch);
  if (threadIdx.x == 0) {
    if (std::is_same<A, double>::value)
      atomicAdd(&st->build_td_d, to_double(bs));
    else
      atomicAdd(reinterpret_cast<unsigned long long*>(&st->build_td_i),
                static_cast<unsigned long long>((long long)bs));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && c >= 0 && c < a.m &&
      KM_INB(st, st->build_step, a.k)) {
    const int step = st->build_step;
    a.med[step] = c;
    a.is_med[c] = 1;
    if (a.gains) a.gains[step] = st->build_gain_d;
    if (a.build_first) {
      st->td_book_d = st->build_gain_d;
      st->td_book_i = st->build_gain_i;
    } else {
      st->td_book_d += st->build_gain_d;
      st->td_book_i += st->build_gain_i;
    }
    st->build_step = step + 1;
  }
}

// ----------------------------------------------- FastPAM2 additional swap
template <class E>
__global__ void __launch_bounds__(kPtThreads) k_fp2_try(const PointArgs a) {
  using T = typename Val<E>::type;  // 16-bit elements widen to int32
  using A = typename Tr<T>::G;   // exact Delta of Eq. (5)
  using R = typename Tr<T>::A;   // removal-loss buffers
  __shared__ A scratch[kPtThreads / 32];
  __shared__ int is_last;
  KmState* st = a.st;
  // The apply kernel that follows accumulates the next removal loss and TD
  // into buffer rb^1; clear it here as the evaluation pass does.
  const int rb = st->rb;
  if (blockIdx.x == 0) {
    R* rnext = static_cast<R*>(a.removal) + (size_t)(rb ^ 1) * a.k_pad;
    for (int i = threadIdx.x; i < a.k; i += blockDim.x) rnext[i] = R(0);
    if (threadIdx.x == 0) static_cast<A*>(a.td2)[rb ^ 1] = A(0);
  }
  if (st->error || st->done) return;
  if (a.fp2_index >= st->fp2_extra) return;
  const int i = a.fp2_order[a.fp2_index];
  if (!KM_INB(st, i, a.k)) return;
  const Key<R> sb = static_cast<const Key<R>*>(a.slot_best)[i];
  const int c = sb.cand;
  if (!KM_INB(st, c, a.m)) return;
  if (a.is_med[c]) {  // already a medoid after an earlier swap
    if (blockIdx.x == 0 && threadIdx.x == 0) st->accept = 0;
    return;
  }
  const int n = a.n;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const E* D = static_cast<const E*>(a.D);
  const T* dn = static_cast<const T*>(a.dn);
  const T* ds = static_cast<const T*>(a.ds);
  A v = A(0);
  if (o < n) {
    const T doc = D[(size_t)c * a.ld + o];
    const T d1 = dn[o], d2 = ds[o];
    if (a.near[o] != i) {
      if (doc < d1) v = dif(doc, d1);          // (c)
    } else {
      v = (doc < d2) ? dif(doc, d1) : dif(d2, d1);  // (b1) / (b2)
    }
  }
  const A bs = block_sum(v, scratch);
  A* parts = static_cast<A*>(a.partials);
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = bs;
    __threadfence();
    is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    A tot = A(0);
    for (int g = 0; g < (int)gridDim.x; ++g) tot += static_cast<volatile A*>(parts)[g];
    const double thr = -a.fp2_tol * st->fp2_dstar;
    if (to_double(tot) < thr) {
      st->accept = 1;
      st->best_d = to_double(tot);
      st->best_i = (long long)tot;
      st->best_slot = i;
      st->best_cand = c;
    } else {
      st->accept = 0;
    }
    st->ticket = 0;
  }
}

// ------------------------------------------------------------- small ones
__global__ void k_mark_medoids(const PointArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.k && KM_INB(a.st, a.med[j], a.m)) a.is_med[a.med[j]] = 1;
}

__global__ void k_fill_medoid_rows(const PointArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < a.m && a.is_med[c]) {
    if (a.cand_delta) a.cand_delta[c] = __longlong_as_double(0x7ff0000000000000ll);
    if (a.cand_slot) a.cand_slot[c] = -1;
  }
}

template <class T>
__global__ void k_removal_to_double(const PointArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rb = a.st->rb;
  if (i < a.k)
    a.out_double[i] =
        Tr<T>::unfx(static_cast<const long long*>(a.removal)[(size_t)rb * a.k_pad + i], a.fshift);
}

// Largest |d| over the matrix (fixes the fixed-point exponent of the SWAP
// sums) and a flag for entries that are negative or not finite.  Float data
// only; one pass over the m x n block (m = n unless bichromatic) with
// 16-byte loads.
__global__ void __launch_bounds__(kPtThreads) k_matrix_scan(const PointArgs a) {
  __shared__ unsigned smax[kPtThreads / 32];
  __shared__ unsigned sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  const float* D = static_cast<const float*>(a.D);
  const int n = a.n;
  const int n4 = (n + 3) >> 2;
  unsigned mx = 0, bad = 0;
  for (long long r = blockIdx.x; r < a.m; r += gridDim.x) {
    const float4* row = reinterpret_cast<const float4*>(D + (size_t)r * a.ld);
    for (int c4 = threadIdx.x; c4 < n4; c4 += blockDim.x) {
      const float4 v = __ldcs(row + c4);
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (4 * c4 + q < n) {
          const unsigned u = __float_as_uint(e[q]);
          // negative (sign bit) or inf/NaN (exponent all ones)
          bad |= (u >> 31) | (((u >> 23) & 0xffu) == 0xffu ? 1u : 0u);
          const unsigned m = u & 0x7fffffffu;
          mx = m > mx ? m : mx;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  if (bad) atomicOr(&sbad, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = max(m, smax[i]);
    atomicMax(&a.scan[0], m);
    if (sbad) atomicOr(&a.scan[1], 1u);
  }
}

// Input check: 32 x 32 tiles (ti, tj) of the upper triangle, each compared
// element by element with its mirror tile (staged in shared memory, so both
// reads are coalesced); diagonal tiles also check d(i, i) = 0.  Float data:
// every entry must be finite and >= 0.
template <class E>
__global__ void __launch_bounds__(256) k_matrix_check(const E* D, long long ld, int n,
                                                      unsigned* flags) {
  __shared__ E mir[32][33];
  const int T = (n + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  unsigned f = 0;
  for (long long L = blockIdx.x; L < (long long)T * T; L += gridDim.x) {
    const int ti = (int)(L / T), tj = (int)(L % T);
    if (tj < ti) continue;  // uniform for the block
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {  // mirror tile: rows of tj, columns of ti
      const int i = tj * 32 + r, j = ti * 32 + tx;
      if (i < n && j < n) mir[r][tx] = D[(size_t)i * ld + j];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = ti * 32 + r, j = tj * 32 + tx;
      if (i < n && j < n) {
        const E v = D[(size_t)i * ld + j];
        const E w = mir[tx][r];  // d(j, i)
        if (memcmp_bits(v, w)) f |= 1u;
        if (i == j && !is_zero(v)) f |= 2u;
        if (bad_value(v)) f |= 4u;
      }
    }
  }
  if (f) atomicOr(flags, f);
}

// ------------------------------------------------------------- launchers
static inline int blocks_for(int n) { return (n + kPtThreads - 1) / kPtThreads; }

cudaError_t launch_cache_init(int dtype, const PointArgs& a, cudaStream_t s) {
  const int grid = blocks_for(a.n_pad);
  const size_t smem = 8 * (size_t)a.k + 8 * (kPtThreads / 32);
  if (dtype == 0) {
    cudaFuncSetAttribute(k_cache_init<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cache_init<int32_t><<<grid, kPtThreads, smem, s>>>(a);
  } else if (dtype == 2) {
    cudaFuncSetAttribute(k_cache_init<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cache_init<uint16_t><<<grid, kPtThreads, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(k_cache_init<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cache_init<float><<<grid, kPtThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(int dtype, const PointArgs& a, cudaStream_t s) {
  const int grid = blocks_for(a.n);
  const size_t smem = 8 * (size_t)a.k + 8 * (kPtThreads / 32);
  if (dtype == 0) {
    cudaFuncSetAttribute(k_apply<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply<int32_t><<<grid, kPtThreads, smem, s>>>(a);
  } else if (dtype == 2) {
    cudaFuncSetAttribute(k_apply<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply<uint16_t><<<grid, kPtThreads, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(k_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply<float><<<grid, kPtThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_commit(int dtype, const PointArgs& a, cudaStream_t s) {
  const int grid = blocks_for(a.n_pad);
  if (dtype == 0)
    k_build_commit<int32_t><<<grid, kPtThreads, 0, s>>>(a);
  else if (dtype == 2)
    k_build_commit<uint16_t><<<grid, kPtThreads, 0, s>>>(a);
  else
    k_build_commit<float><<<grid, kPtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fp2_try(int dtype, const PointArgs& a, cudaStream_t s) {
  const int grid = blocks_for(a.n);
  if (grid > kMaxGrid) return cudaErrorInvalidConfiguration;
  if (dtype == 0)
    k_fp2_try<int32_t><<<grid, kPtThreads, 0, s>>>(a);
  else if (dtype == 2)
    k_fp2_try<uint16_t><<<grid, kPtThreads, 0, s>>>(a);
  else
    k_fp2_try<float><<<grid, kPtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// A fresh state record (every field zero, no last swap, the caller's wait
// limit), written on the device so that resetting it does not synchronise
// the host with the stream.
__global__ void k_reset_state(KmState* st, unsigned long long wait_ns) {
  unsigned* w = reinterpret_cast<unsigned*>(st);
  for (int i = threadIdx.x; i < (int)(sizeof(KmState) / 4); i += blockDim.x) w[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->last = -1;
    st->wait_ns = wait_ns;
  }
}

cudaError_t launch_reset_state(KmState* st, unsigned long long wait_ns, cudaStream_t s) {
  k_reset_state<<<1, 128, 0, s>>>(st, wait_ns);
  return cudaGetLastError();
}

// The BUILD -> SWAP hand-off of kmedoids_run: keeps the state record as the
// BUILD left it (its step count, bookkept TD and any recorded failure) for
// the one read at the end of the call, before the SWAP resets the record.
// After a failed BUILD the medoid slots are set to 0 .. k-1 so that the SWAP
// kernels, which run regardless, index valid rows; the call then reports the
// BUILD's failure.
__global__ void k_build_handoff(KmState* st, KmState* saved, int32_t* med, int k) {
  const unsigned* w = reinterpret_cast<const unsigned*>(st);
  unsigned* o = reinterpret_cast<unsigned*>(saved);
  for (int i = threadIdx.x; i < (int)(sizeof(KmState) / 4); i += blockDim.x) o[i] = w[i];
  if (st->error)
    for (int j = threadIdx.x; j < k; j += blockDim.x) med[j] = j;
}

cudaError_t launch_build_handoff(KmState* st, KmState* saved, int32_t* med, int k,
                                 cudaStream_t s) {
  k_build_handoff<<<1, 128, 0, s>>>(st, saved, med, k);
  return cudaGetLastError();
}

// The condition of the FastPAM1 SWAP loop graph, evaluated after each pass
// and its swap: run another body while the loop has not converged, no
// kernel reported an error and fewer than max_iter passes ran.  A guard
// counted here alone ends the loop after max_iter bodies whatever the other
// kernels did.
__global__ void k_swap_loop_cond(KmState* st, cudaGraphConditionalHandle h, int max_iter) {
  const int g = ++st->loop_guard;
  const bool more = !st->done && !st->error && st->iter < max_iter && g < max_iter;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

cudaError_t launch_swap_loop_cond(KmState* st, unsigned long long handle, int max_iter,
                                  cudaStream_t s) {
  k_swap_loop_cond<<<1, 1, 0, s>>>(st, (cudaGraphConditionalHandle)handle, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_mark_medoids(const PointArgs& a, cudaStream_t s) {
  k_mark_medoids<<<(a.k + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fill_medoid_rows(const PointArgs& a, cudaStream_t s) {
  k_fill_medoid_rows<<<blocks_for(a.m), kPtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_removal_to_double(int dtype, const PointArgs& a, cudaStream_t s) {
  if (dtype == 0 || dtype == 2)
    k_removal_to_double<int32_t><<<(a.k + 255) / 256, 256, 0, s>>>(a);
  else
    k_removal_to_double<float><<<(a.k + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_matrix_check(int dtype, const void* D, long long ld, int n, unsigned* flags,
                                cudaStream_t s) {
  long long tiles = (long long)((n + 31) / 32) * ((n + 31) / 32);
  int grid = device_sm_count() * 8;
  if (grid < 1) grid = 1;
  if (tiles < grid) grid = (int)tiles;
  if (dtype == 0)
    k_matrix_check<int32_t><<<grid, 256, 0, s>>>(static_cast<const int32_t*>(D), ld, n, flags);
  else if (dtype == 2)
    k_matrix_check<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(D), ld, n, flags);
  else
    k_matrix_check<float><<<grid, 256, 0, s>>>(static_cast<const float*>(D), ld, n, flags);
  return cudaGetLastError();
}

cudaError_t launch_matrix_scan(const PointArgs& a, cudaStream_t s) {
  int grid = device_sm_count() * 4;
  if (grid < 1) grid = 1;
  if (grid > a.m) grid = a.m;
  k_matrix_scan<<<grid, kPtThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int device_sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return v;
}

}  // namespace km

// km_batched.cu -- many independent PAM instances in one persistent launch,
// and CLARA (Sec. 2.1; FastCLARA, Sec. 3.4) on top of it.
//
// k_batch_pam: each CTA takes instances from an atomic queue (ordered
// largest first) and runs the whole method on one instance: BUILD (Alg. 1)
// or the caller's starting medoids (restarts from random starts), the exact
// per-point cache, and FastPAM1 SWAP (Alg. 3, Eq. (7)) or the eager
// FasterPAM (Alg. 4) to convergence, with every per-point quantity in shared
// memory and one warp per candidate row.  Float sums of the SWAP pass use the same
// exact 64-bit fixed point as the single-instance kernels (scale from the
// instance's largest entry, found during BUILD step 0).  Instances need
// n <= 4096 and k <= 128.
//
// CLARA: the caller passes the sample indices (drawn by its own generator);
// the sample matrices are built with the FP64 recipe below, solved as extra
// instances of k_batch_pam, then every point of the full data set is
// assigned to each sample's medoids (FP32 direct differences, FP64 TD sum)
// and the sample with the least TD wins (lowest index on ties).
#define KM_SRC_ID 6  // names this file in bounds-check reports
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"

namespace km {

constexpr int kBatchMaxN = 4096;
constexpr int kBatchMaxK = 128;
constexpr int kBatchMaxCount = 65535;  // also the grid height of the distance kernel
constexpr int kDistMaxDim = 864;       // 64 staged points + the tile fit in shared memory

// Instances 0 .. count_a - 1 come from the first table (arena, inst,
// medoids, out), instances count_a .. count - 1 from the second (arena2,
// inst2, medoids2, out2; CLARA's samples when a batch and CLARA share one
// launch).
struct BatchArgs {
  const float* arena;
  const km_instance* inst;
  int count;                 // both tables
  int count_a;               // the first table
  const int32_t* order;      // instance processing order (largest first)
  int32_t* medoids;          // concatenated, at inst[i].medoid_offset
  km_batch_result* out;
  const float* arena2;
  const km_instance* inst2;
  int32_t* medoids2;
  km_batch_result* out2;
  unsigned* queue;           // next position in order
  int* error;
  int max_iter;
  double tol;
  int start_given;           // 1: start from the medoids in `medoids` (no BUILD)
  int eager;                 // 1: FasterPAM (Alg. 4) instead of FastPAM1
};

// Euclidean matrix of m points: FP64 differences, squares accumulated with
// fused multiply-adds in coordinate order, FP64 square root, one rounding to
// FP32.  Instance/sample q has points P[idx[q][i]] (idx may be NULL:
// consecutive points from point_off[q]) and writes rows of ld elements at
// D + d_off[q] (zeros in the padding columns).
struct DistArgs {
  const float* P;
  int dim;
  const long long* point_off;  // per instance: first point (idx == NULL)
  const int32_t* idx;          // per instance sample indices (s each)
  int s;
  const km_instance* inst;
  float* D;
  int count;
};

__device__ __forceinline__ double dist_fp64(const float* xi, const float* xj, int dim) {
  double sq = 0.0;
  for (int t = 0; t < dim; ++t) {
    const double df = (double)xi[t] - (double)xj[t];
    sq = __fma_rn(df, df, sq);
  }
  return sqrt(sq);
}

// 32 x 32 tiles of the upper triangle, each written with its mirror image:
// d(j, i) squares the negated differences of d(i, j), so the recipe gives
// bitwise-symmetric values and half the FP64 work suffices.  The 64 points
// of a tile are staged in shared memory (row stride dim | 1 words, so the
// 32 lanes reading 32 different points hit distinct banks).
__global__ void __launch_bounds__(256) k_batch_dist(const DistArgs a) {
  extern __shared__ float xsm[];  // [64][stride]
  __shared__ float tile[32][33];
  const int q = blockIdx.y;
  if (q >= a.count) return;
  const km_instance in = a.inst[q];
  float* D = a.D + in.offset;
  const int m = in.n, dim = a.dim, stride = dim | 1;
  const int T = (m + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (long long L = blockIdx.x; L < (long long)T * T; L += gridDim.x) {
    const int ti = (int)(L / T), tj = (int)(L % T);
    if (tj < ti) continue;  // the block's uniform choice
    __syncthreads();        // the previous tile's reads of xsm / tile are done
    for (int e = threadIdx.x; e < 64 * dim; e += blockDim.x) {
      const int r = e / dim, t = e % dim;
      const int gi = (r < 32) ? ti * 32 + r : tj * 32 + (r - 32);
      float v = 0.f;
      if (gi < m) {
        const long long pt = a.idx ? a.idx[(long long)q * a.s + gi] : a.point_off[q] + gi;
        v = a.P[pt * dim + t];
      }
      xsm[r * stride + t] = v;
    }
    __syncthreads();
    const float* xj = xsm + (32 + tx) * stride;
    const int j = tj * 32 + tx;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int ii = ty + 8 * r, i = ti * 32 + ii;
      const float v = (float)dist_fp64(xsm + ii * stride, xj, dim);
      if (i < m && j < m) D[(size_t)i * in.ld + j] = v;
      tile[ii][tx] = v;
    }
    if (ti != tj) {
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int jj = ty + 8 * r;
        const int i2 = ti * 32 + tx, j2 = tj * 32 + jj;
        if (i2 < m && j2 < m) D[(size_t)j2 * in.ld + i2] = tile[tx][jj];
      }
    }
  }
  const int pad = in.ld - m;
  if (pad > 0)
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * pad;
         e += (long long)gridDim.x * blockDim.x)
      D[(size_t)(e / pad) * in.ld + m + (int)(e % pad)] = 0.f;
}

size_t dist_smem(int dim) { return 4 * (size_t)64 * (size_t)(dim | 1); }

// Processing order, largest work first (n^2 (k + 1), the BUILD plus SWAP
// passes' scale): the rank of instance i is the number of instances with
// more work, or equal work and a lower index, i.e. a stable sort by counting.
__device__ __forceinline__ double batch_work(const km_instance& a) {
  return (double)a.n * (double)a.n * (double)(a.k + 1);
}

// Instance i of the two tables (i < count_a: the first).
__device__ __forceinline__ km_instance inst_at(const km_instance* ia, int count_a,
                                              const km_instance* ib, int i) {
  return i < count_a ? ia[i] : ib[i - count_a];
}

__global__ void __launch_bounds__(256) k_batch_order(const km_instance* inst, int count_a,
                                                     const km_instance* inst2, int count,
                                                     int32_t* order) {
  __shared__ double w[256];
  for (int i0 = blockIdx.x * blockDim.x; i0 < count; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + threadIdx.x;
    const double wi = (i < count) ? batch_work(inst_at(inst, count_a, inst2, i)) : 0.0;
    int r = 0;
    for (int j0 = 0; j0 < count; j0 += 256) {
      __syncthreads();
      if (j0 + threadIdx.x < count)
        w[threadIdx.x] = batch_work(inst_at(inst, count_a, inst2, j0 + threadIdx.x));
      __syncthreads();
      const int m = min(256, count - j0);
      for (int t = 0; t < m; ++t) {
        const double wj = w[t];
        r += (wj > wi || (wj == wi && j0 + t < i)) ? 1 : 0;
      }
    }
    if (i < count) order[r] = i;
  }
}

// Per-warp cp.async ring: every warp streams its own candidate rows through
// STAGES stages of 512 columns (32 lanes x 4 float4), so each SM keeps up
// to WARPS x (STAGES - 1) x 2 KB of row data in flight.  (One 1-D
// bulk copy per stage issued by lane 0, with an mbarrier per stage, measured
// 14 % slower on GB300 than these per-lane 16-byte copies.)
constexpr int kRingFloats = 512;

// dn, ds and the ring are read as float4: keep them 16-byte aligned.
template <int WARPS, int STAGES>
struct BatchSmem {
  alignas(16) float ring[WARPS][STAGES][kRingFloats];
  alignas(16) float dn[kBatchMaxN];
  alignas(16) float ds[kBatchMaxN];
  uint8_t near[kBatchMaxN];
  uint8_t sec[kBatchMaxN];
  uint8_t is_med[kBatchMaxN];
  int32_t med[kBatchMaxK];
  long long rl[kBatchMaxK];
  long long acc[WARPS][kBatchMaxK];
  double wd[WARPS];
  long long wl[WARPS];
  int wslot[WARPS];
  int wcand[WARPS];
  unsigned wmax[WARPS];
  int inst;
  int cstar;
  int istar;
  double dstar;
  long long dstar_i;
};

// The geometries of the persistent kernel (warps per CTA, ring stages), as
// numbered by km_options.tune for the batched form (tune 0 = entry 1).
#define KM_BATCH_GEOMETRIES(X) X(1, 16, 4) X(2, 8, 4) X(3, 16, 3) X(4, 8, 8) X(5, 12, 5)
constexpr int kBatchGeometries = 5;
#define KM_BATCH_ALIGN(G, W, S)                                                          \
  using BatchSmemG##G = BatchSmem<W, S>;                                                 \
  static_assert(offsetof(BatchSmemG##G, dn) % 16 == 0 &&                                 \
                    offsetof(BatchSmemG##G, ds) % 16 == 0,                               \
                "float4 reads of d_n / d_s need 16-byte alignment");                      \
  static_assert(sizeof(BatchSmemG##G) <= 227 * 1024, "shared memory of one CTA");
KM_BATCH_GEOMETRIES(KM_BATCH_ALIGN)
#undef KM_BATCH_ALIGN

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// FP32 (hi, lo) pair sum across the warp with error-free TwoSum; FP64 out.
__device__ __forceinline__ double warp_sum_pair(float hi, float lo) {
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
  return (double)hi + (double)lo;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Streams the warp's candidate rows c = warp, warp + WARPS, ... (medoid rows
// skipped) through the warp's ring.  on_chunk(c, o, v, stage) receives the
// lane's entries row[o + 128 u + 4 lane + t] as v[u].t (entries at or beyond
// n are stale and must be masked by the caller) and a pointer to the stage;
// on_row_end(c) runs once per row.  Both are warp-uniform.  Each lane reads
// back only the 16-byte pieces it copied itself, so cp.async.wait_group is the
// only synchronisation; it completes when the lane's own copies land.
template <int WARPS, int STAGES, class Chunk, class RowEnd>
__device__ __forceinline__ void stream_rows(BatchSmem<WARPS, STAGES>& S, const float* D, int n, int ld,
                                            int warp, int lane, Chunk&& on_chunk,
                                            RowEnd&& on_row_end) {
  float(*ring)[kRingFloats] = S.ring[warp];
  int ic = warp;
  while (ic < n && S.is_med[ic]) ic += WARPS;
  int io = 0;
  int cc = ic, co = 0;
  auto issue = [&](int slot) {
    if (ic < n) {
      const float* row = D + (size_t)ic * ld;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = io + 128 * u + 4 * lane;
        if (p < n) cp_async16(&ring[slot][128 * u + 4 * lane], row + p);
      }
      io += kRingFloats;
      if (io >= n) {
        io = 0;
        ic += WARPS;
        while (ic < n && S.is_med[ic]) ic += WARPS;
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) issue(s);
  int slot = 0;
  while (cc < n) {
    issue(slot == 0 ? STAGES - 1 : slot - 1);
    cp_async_wait<STAGES - 1>();
    const float* stage = ring[slot];
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(stage + 128 * u + 4 * lane);
    on_chunk(cc, co, v, stage);
    co += kRingFloats;
    if (co >= n) {
      on_row_end(cc);
      co = 0;
      cc += WARPS;
      while (cc < n && S.is_med[cc]) cc += WARPS;
    }
    slot = (slot + 1 == STAGES) ? 0 : slot + 1;
  }
  cp_async_wait<0>();
}

// Streams one row (n entries) through the warp's ring, as stream_rows does
// for a sequence of rows: on_chunk(o, v, stage) for column chunks o = 0,
// 512, ...; entries at or beyond n are stale and masked by the caller.
template <int WARPS, int STAGES, class Chunk>
__device__ __forceinline__ void stream_one_row(BatchSmem<WARPS, STAGES>& S, const float* row, int n,
                                               int warp, int lane, Chunk&& on_chunk) {
  float(*ring)[kRingFloats] = S.ring[warp];
  const int nch = (n + kRingFloats - 1) / kRingFloats;
  auto issue = [&](int j) {
    if (j < nch) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = j * kRingFloats + 128 * u + 4 * lane;
        if (p < n) cp_async16(&ring[j % STAGES][128 * u + 4 * lane], row + p);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int j = 0; j < STAGES - 1; ++j) issue(j);
  for (int j = 0; j < nch; ++j) {
    issue(j + STAGES - 1);
    cp_async_wait<STAGES - 1>();
    const float* stage = ring[j % STAGES];
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(stage + 128 * u + 4 * lane);
    on_chunk(j * kRingFloats, v, stage);
  }
  cp_async_wait<0>();
}

// floor(x * 2^f) for finite x >= 0 with 2^f = s1 * s2 (each a normal power
// of two), equal to the integer-only fx_of.  y = x * 2^f is exact in FP32
// (power-of-two scaling; below the normal range both the rounded and the
// exact value floor to 0) and y < 2^62 by the choice of f.  The 64-bit
// result is assembled from two 32-bit conversions (a 64-bit conversion runs
// on GB300's narrow FP64 pipe): hi = floor(y / 2^32) (exact scaling; hi is
// either below 2^24 or y / 2^32 itself, so it converts back to FP32
// exactly), r = y - hi * 2^32 in one fused operation (exact: r < 2^32 and a
// multiple of y's unit in the last place), lo = floor(r).
__device__ __forceinline__ long long fx_scaled(float x, float s1, float s2) {
  const float y = (x * s1) * s2;
  const unsigned hi = __float2uint_rz(y * 0x1p-32f);
  const float r = __fmaf_rn(-(float)hi, 0x1p32f, y);
  const unsigned lo = __float2uint_rd(r);
  return (long long)(((unsigned long long)hi << 32) | lo);
}

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ float f4get(const float4& v, int t) {
  return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}

template <int WARPS, int STAGES>
__global__ void __launch_bounds__(WARPS * 32, 1) k_batch_pam(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<WARPS, STAGES>& S = *reinterpret_cast<BatchSmem<WARPS, STAGES>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NT = WARPS * 32;

  while (true) {
    if (tid == 0) {
      const unsigned p = atomicAdd(a.queue, 1u);
      S.inst = (p < (unsigned)a.count) ? a.order[p] : -1;
    }
    __syncthreads();
    const int q = S.inst;
    if (q < 0) break;
    const bool first = q < a.count_a;
    const km_instance in = first ? a.inst[q] : a.inst2[q - a.count_a];
    const int n = in.n, k = in.k, ld = in.ld;
    const float* D = (first ? a.arena : a.arena2) + in.offset;
    km_batch_result* outq = first ? a.out + q : a.out2 + (q - a.count_a);
    int32_t* medq = (first ? a.medoids : a.medoids2) + in.medoid_offset;
    km_batch_result res;
    res.td = 0.0;
    res.iterations = 0;
    res.swaps = 0;
    res.status = 0;
    res.pad = 0;
    if (n < 1 || n > kBatchMaxN || k < 1 || k > kBatchMaxK || k > n || ld < n || (ld & 3) ||
        (in.offset & 3) || in.offset < 0) {
      if (tid == 0) {
        res.status = KM_E_INVALID;
        *outq = res;
      }
      __syncthreads();
      continue;
    }
    // d_n and d_s of the columns past n up to the ring's 512-column stride
    // hold -inf, so `d < d_n` and `d < d_s` never hold there and the stream
    // loops need no column bounds checks after BUILD step 0
    const int npad = (n + kRingFloats - 1) / kRingFloats * kRingFloats;
    for (int o = tid; o < npad; o += NT) {
      if (o < n) {
        S.is_med[o] = 0;
      } else {
        S.dn[o] = -__int_as_float(0x7f800000);
        S.ds[o] = -__int_as_float(0x7f800000);
      }
    }
    __syncthreads();

    unsigned mloc = 0;
    if (a.start_given) {
      // the largest entry over the whole matrix (fixed-point scale of the
      // SWAP sums), streamed with no row marked as a medoid yet
      stream_rows<WARPS, STAGES>(
          S, D, n, ld, warp, lane,
          [&](int, int o, const float4(&v)[4], const float*) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int p0 = o + 128 * u + 4 * lane;
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (p0 + t < n) mloc = max(mloc, __float_as_uint(f4get(v[u], t)) & 0x7fffffffu);
            }
          },
          [&](int) {});
      for (int o = 16; o > 0; o >>= 1) mloc = max(mloc, __shfl_xor_sync(0xffffffffu, mloc, o));
      if (lane == 0) S.wmax[warp] = mloc;
      // the caller's starting medoids must be in range and distinct
      if (tid == 0) {
        int bad = 0;
        for (int j = 0; j < k && !bad; ++j) {
          const int m = medq[j];
          if (m < 0 || m >= n || S.is_med[m]) {
            bad = 1;
          } else {
            S.is_med[m] = 1;
            S.med[j] = m;
          }
        }
        S.cstar = bad;
      }
      __syncthreads();
      if (S.cstar) {
        if (tid == 0) {
          res.status = KM_E_INVALID;
          *outq = res;
        }
        __syncthreads();
        continue;
      }
    }

    // ------------------------------------------------------------- BUILD
    for (int step = 0; step < (a.start_given ? 0 : k); ++step) {
      double bd = 1e300;
      int bc = INT_MAX;
      float hs = 0.f, hc = 0.f, hs2 = 0.f, hc2 = 0.f;  // two compensated chains
      stream_rows<WARPS, STAGES>(
          S, D, n, ld, warp, lane,
          [&](int, int o, const float4(&v)[4], const float*) {
            if (step == 0) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int p0 = o + 128 * u + 4 * lane;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  if (p0 + t < n) {
                    const float e = f4get(v[u], t);
                    mloc = max(mloc, __float_as_uint(e) & 0x7fffffffu);
                    kahan_add(hs, hc, e);
                  }
                }
              }
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int p0 = o + 128 * u + 4 * lane;  // < npad <= kBatchMaxN
                const float4 d4 = *reinterpret_cast<const float4*>(&S.dn[p0]);
                // min(e - d_n, 0): e - d_n is negative exactly when e < d_n
                // (and +inf on the -inf padding, giving 0)
                kahan_add(hs, hc, fminf(v[u].x - d4.x, 0.f));
                kahan_add(hs2, hc2, fminf(v[u].y - d4.y, 0.f));
                kahan_add(hs, hc, fminf(v[u].z - d4.z, 0.f));
                kahan_add(hs2, hc2, fminf(v[u].w - d4.w, 0.f));
              }
            }
          },
          [&](int c) {
            // fold the two chains with TwoSum, then across the warp
            const float sh = hs + hs2;
            const float bp = sh - hs;
            const float err = (hs - (sh - bp)) + (hs2 - bp);
            const double g = warp_sum_pair(sh, err - hc - hc2);
            hs = hc = hs2 = hc2 = 0.f;
            if (g < bd) {  // rows visited in ascending order: keeps the lowest c
              bd = g;
              bc = c;
            }
          });
      if (lane == 0) {
        S.wd[warp] = bd;
        S.wcand[warp] = bc;
      }
      if (step == 0) {
        for (int o = 16; o > 0; o >>= 1) mloc = max(mloc, __shfl_xor_sync(0xffffffffu, mloc, o));
        if (lane == 0) S.wmax[warp] = mloc;
      }
      __syncthreads();
      if (tid == 0) {
        double b = S.wd[0];
        int c = S.wcand[0];
        for (int w = 1; w < WARPS; ++w)
          if (S.wd[w] < b || (S.wd[w] == b && S.wcand[w] < c)) {
            b = S.wd[w];
            c = S.wcand[w];
          }
        S.cstar = c;
        S.med[step] = c;
        S.is_med[c] = 1;
        S.dstar = (step == 0) ? b : S.dstar + b;  // bookkept TD
      }
      __syncthreads();
      const int c = S.cstar;
      const float* row = D + (size_t)c * ld;
      for (int o = tid; o < n; o += NT) {
        const float v = row[o];
        S.dn[o] = (step == 0 || v < S.dn[o]) ? v : S.dn[o];
      }
      __syncthreads();
    }

    // fixed-point exponent from the largest entry and n (as the grid path)
    unsigned mbits = 0;
    for (int w = 0; w < WARPS; ++w) mbits = max(mbits, S.wmax[w]);
    int em = 0;
    {
      const float mf = __uint_as_float(mbits);
      if (mf > 0.f) em = ilogbf(mf) + 1;  // mf < 2^em
    }
    int bn = 0;
    while ((1ll << bn) <= (long long)n) ++bn;
    const int f = 60 - bn - em;
    // 2^f split in two normal factors: -81 <= f <= 209 for finite data
    const float fs1 = pow2f(f / 2), fs2 = pow2f(f - f / 2);

    // --------------------------------------------- cache, removal loss, TD
    // nearest slot, d_n and d_s of every point from the k medoid rows (read
    // column-wise, eight rows in flight); lowest slot among equal distances
    auto cache_all = [&]() {
      for (int i = tid; i < k; i += NT) S.rl[i] = 0;
      __syncthreads();
      for (int o = tid; o < n; o += NT) {
        int n1 = -1, n2 = -1;
        float d1 = 0.f, d2 = 0.f;
        for (int j0 = 0; j0 < k; j0 += 8) {
          float v8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            v8[u] = (j0 + u < k) ? D[(size_t)S.med[j0 + u] * ld + o] : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (j0 + u < k) {
              const float v = v8[u];
              if (n1 < 0 || v < d1) {
                n2 = n1;
                d2 = d1;
                n1 = j0 + u;
                d1 = v;
              } else if (n2 < 0 || v < d2) {
                n2 = j0 + u;
                d2 = v;
              }
            }
          }
        }
        S.near[o] = (uint8_t)n1;
        S.sec[o] = (uint8_t)(n2 < 0 ? 0 : n2);
        S.dn[o] = d1;
        S.ds[o] = (n2 < 0) ? __int_as_float(0x7f800000) : d2;
        if (n2 >= 0) atomic_add_shared64(&S.rl[n1], fx_of(d2, f) - fx_of(d1, f));
      }
      __syncthreads();
    };

    if (k < n && k >= 2 && a.eager) {
      // ------------------------------------------- FasterPAM (Alg. 4)
      // windows of WARPS scan positions, one candidate row per warp against
      // the current medoids; the first improving position is applied at
      // once (incremental cache update) and the next window starts after
      // it, so the decisions are those of the sequential scan
      cache_all();
      long long pos = 0, last = -1;
      bool conv = false;
      const long long pos_limit = (long long)a.max_iter * n;
      // acceptance Delta < -tol on the fixed-point sums: Delta 2^f < -tol 2^f
      // (exact power-of-two scaling; evaluated once, FP64 is slow here)
      const double inv_scale = exp2(-(double)f);
      const double accept_below = -a.tol * exp2((double)f);
      while (pos < pos_limit) {
        const long long stop = (last < 0) ? (long long)n : last + n;
        const long long wlen = min((long long)WARPS, stop - pos);
        long long tot = LLONG_MAX;
        int bi = -1;
        const int c = (warp < wlen) ? (int)((pos + warp) % n) : -1;
        if (c >= 0 && !S.is_med[c]) {
          long long* ar = S.acc[warp];
          for (int i = lane; i < k; i += 32) ar[i] = 0;
          __syncwarp();
          long long lp = 0;
          stream_one_row<WARPS, STAGES>(S, D + (size_t)c * ld, n, warp, lane,
                                [&](int o, const float4(&v)[4], const float* stage) {
            unsigned mask = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int p0 = o + 128 * u + 4 * lane;  // < npad <= kBatchMaxN
              const float4 s4 = *reinterpret_cast<const float4*>(&S.ds[p0]);
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (f4get(v[u], t) < f4get(s4, t)) mask |= 1u << (4 * u + t);
            }
            while (mask) {
              const int b = __ffs(mask) - 1;
              mask &= mask - 1;
              const int col = 128 * (b >> 2) + 4 * lane + (b & 3);
              const int p = o + col;
              const float e = stage[col];
              const float dnp = S.dn[p], dsp = S.ds[p];
              const int sl = S.near[p];
              const long long xd = fx_scaled(e, fs1, fs2), xs = fx_scaled(dsp, fs1, fs2);
              if (e < dnp) {
                const long long xn = fx_scaled(dnp, fs1, fs2);
                lp += xd - xn;
                atomic_add_shared64(&ar[sl], xn - xs);
              } else {
                atomic_add_shared64(&ar[sl], xd - xs);
              }
            }
          });
          __syncwarp();
          long long bv = LLONG_MAX;
          for (int i = lane; i < k; i += 32) {
            const long long v = S.rl[i] + ar[i];
            if (v < bv) {
              bv = v;
              bi = i;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) {
              bv = ov;
              bi = oi;
            }
          }
          tot = bv + warp_sum(lp);
        }
        if (lane == 0) {
          S.wl[warp] = tot;
          S.wslot[warp] = (c >= 0 && !S.is_med[c]) ? bi : -1;
        }
        __syncthreads();
        if (tid == 0) {
          int fw = -1;
          for (int w = 0; w < (int)wlen; ++w)
            if (S.wslot[w] >= 0 &&
                (a.tol == 0.0 ? S.wl[w] < 0 : (double)S.wl[w] < accept_below)) {
              fw = w;
              break;
            }
          S.cstar = (fw >= 0) ? (int)((pos + fw) % n) : -1;
          S.istar = (fw >= 0) ? S.wslot[fw] : -1;
          S.dstar_i = (fw >= 0) ? S.wl[fw] : 0;
          S.wcand[0] = fw;
        }
        __syncthreads();
        const int fw = S.wcand[0];
        if (fw < 0) {
          pos += wlen;
          if (pos >= stop) {
            conv = true;
            break;
          }
          continue;
        }
        last = pos + fw;
        pos = last + 1;
        // ------------------------------------------- apply (incremental)
        const int i_s = S.istar, c_s = S.cstar;
        const float* rowc = D + (size_t)c_s * ld;
        __syncthreads();  // every thread has read istar / cstar
        if (tid == 0) {
          S.is_med[S.med[i_s]] = 0;
          S.med[i_s] = c_s;
          S.is_med[c_s] = 1;
          S.dstar += (double)S.dstar_i * inv_scale;
        }
        for (int i = tid; i < k; i += NT) S.rl[i] = 0;
        __syncthreads();
        // the new medoid's distances to this thread's points, all in flight
        // before any is used (most points need only this one)
        constexpr int kPer = (kBatchMaxN + NT - 1) / NT;
        float dcv[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int o = tid + u * NT;
          dcv[u] = (o < n) ? rowc[o] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int o = tid + u * NT;
          if (o >= n) break;
          int n1 = S.near[o], n2 = S.sec[o];
          float d1 = S.dn[o], d2 = S.ds[o];
          if (n1 == i_s || n2 == i_s) {
            // the removed medoid was nearest or second: rescan every slot
            // (eight medoid rows in flight)
            n1 = -1;
            n2 = -1;
            for (int j0 = 0; j0 < k; j0 += 8) {
              float v8[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                v8[u] = (j0 + u < k) ? D[(size_t)S.med[j0 + u] * ld + o] : 0.f;
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (j0 + u < k) {
                  const float v = v8[u];
                  if (n1 < 0 || v < d1) {
                    n2 = n1;
                    d2 = d1;
                    n1 = j0 + u;
                    d1 = v;
                  } else if (n2 < 0 || v < d2) {
                    n2 = j0 + u;
                    d2 = v;
                  }
                }
              }
            }
          } else {
            // only the new medoid enters: top-2 of {nearest, second, new}
            const float dc = dcv[u];
            if (dc < d1 || (dc == d1 && i_s < n1)) {
              n2 = n1;
              d2 = d1;
              n1 = i_s;
              d1 = dc;
            } else if (dc < d2 || (dc == d2 && i_s < n2)) {
              n2 = i_s;
              d2 = dc;
            }
          }
          S.near[o] = (uint8_t)n1;
          S.sec[o] = (uint8_t)n2;
          S.dn[o] = d1;
          S.ds[o] = d2;
          atomic_add_shared64(&S.rl[n1], fx_of(d2, f) - fx_of(d1, f));
        }
        ++res.swaps;
        __syncthreads();
      }
      res.iterations = (int)((pos + n - 1) / n);
      res.status = conv ? 0 : KM_E_NOT_CONVERGED;
    } else if (k < n) {
      cache_all();
      int it = 0;
      bool conv = false;
      while (it < a.max_iter) {
        // ----------------------------------------------- SWAP evaluation
        long long wbest = LLONG_MAX;
        int wslot = INT_MAX, wcand = INT_MAX;
        if (k >= 2) {
          long long* ar = S.acc[warp];
          for (int i = lane; i < k; i += 32) ar[i] = 0;
          __syncwarp();
          long long lp = 0;  // this lane's part of the shared accumulator
          stream_rows<WARPS, STAGES>(
              S, D, n, ld, warp, lane,
              [&](int, int o, const float4(&v)[4], const float* stage) {
                // fast path: one d < d_s test per entry; hits in a lane mask
                unsigned mask = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int p0 = o + 128 * u + 4 * lane;  // < npad <= kBatchMaxN
                  const float4 s4 = *reinterpret_cast<const float4*>(&S.ds[p0]);
#pragma unroll
                  for (int t = 0; t < 4; ++t)
                    if (f4get(v[u], t) < f4get(s4, t)) mask |= 1u << (4 * u + t);
                }
                // each lane walks its own hits (Eq. (7) cases); a warp-wide
                // compaction of the hits measured slower on GB300
                while (mask) {
                  const int b = __ffs(mask) - 1;
                  mask &= mask - 1;
                  const int col = 128 * (b >> 2) + 4 * lane + (b & 3);
                  const int p = o + col;
                  const float e = stage[col];
                  const float dnp = S.dn[p], dsp = S.ds[p];
                  const int sl = S.near[p];
                  const long long xd = fx_scaled(e, fs1, fs2), xs = fx_scaled(dsp, fs1, fs2);
                  if (e < dnp) {
                    const long long xn = fx_scaled(dnp, fs1, fs2);
                    lp += xd - xn;
                    atomic_add_shared64(&ar[sl], xn - xs);
                  } else {
                    atomic_add_shared64(&ar[sl], xd - xs);
                  }
                }
              },
              [&](int c) {
                __syncwarp();
                long long bv = LLONG_MAX;
                int bi = INT_MAX;
                for (int i = lane; i < k; i += 32) {
                  const long long v = S.rl[i] + ar[i];
                  if (v < bv) {
                    bv = v;
                    bi = i;
                  }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                  const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
                  const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                  if (ov < bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                  }
                }
                const long long tot = bv + warp_sum(lp);
                lp = 0;
                if (tot < wbest || (tot == wbest && (bi < wslot || (bi == wslot && c < wcand)))) {
                  wbest = tot;
                  wslot = bi;
                  wcand = c;
                }
                __syncwarp();
                for (int i = lane; i < k; i += 32) ar[i] = 0;
                __syncwarp();
              });
        } else {
          // k = 1: the best single swap is the 1-medoid (Eq. (3))
          for (int c = warp; c < n; c += WARPS) {
            if (S.is_med[c]) continue;
            const float* row = D + (size_t)c * ld;
            long long s = 0;
            for (int o = lane; o < n; o += 32) s += fx_of(row[o], f) - fx_of(S.dn[o], f);
            s = warp_sum(s);
            if (s < wbest || (s == wbest && c < wcand)) {
              wbest = s;
              wslot = 0;
              wcand = c;
            }
          }
        }
        if (lane == 0) {
          S.wl[warp] = wbest;
          S.wslot[warp] = wslot;
          S.wcand[warp] = wcand;
        }
        __syncthreads();
        if (tid == 0) {
          long long b = S.wl[0];
          int bs = S.wslot[0], bc = S.wcand[0];
          for (int w = 1; w < WARPS; ++w) {
            const long long v = S.wl[w];
            if (v < b || (v == b && (S.wslot[w] < bs || (S.wslot[w] == bs && S.wcand[w] < bc)))) {
              b = v;
              bs = S.wslot[w];
              bc = S.wcand[w];
            }
          }
          S.dstar_i = b;
          S.istar = bs;
          S.cstar = bc;
        }
        __syncthreads();
        ++it;
        const long long b = S.dstar_i;
        const int bs = S.istar, bc = S.cstar;
        if (bc == INT_MAX || !((double)b * exp2(-(double)f) < -a.tol)) {
          conv = true;
          break;
        }
        // --------------------------------------------------------- apply
        if (tid == 0) {
          S.is_med[S.med[bs]] = 0;
          S.med[bs] = bc;
          S.is_med[bc] = 1;
          S.dstar += (double)b * exp2(-(double)f);
        }
        ++res.swaps;
        __syncthreads();
        cache_all();
      }
      res.iterations = it;
      res.status = conv ? 0 : KM_E_NOT_CONVERGED;
    } else {
      // k = n: every point is a medoid
      for (int o = tid; o < n; o += NT) S.dn[o] = 0.f;
      __syncthreads();
      res.iterations = 1;
    }
    // exact TD of the result (FP64) and outputs
    double tdl = 0.0;
    for (int o = tid; o < n; o += NT) tdl += (double)S.dn[o];
    tdl = warp_sum(tdl);
    if (lane == 0) S.wd[warp] = tdl;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < WARPS; ++w) t += S.wd[w];
      res.td = t;
      *outq = res;
    }
    for (int j = tid; j < k; j += NT) medq[j] = S.med[j];
    __syncthreads();
  }
}

// CLARA sample q as a batch instance: s rows of ld elements at q s ld in the
// sample arena, k medoids at q k.
__global__ void k_clara_inst(km_instance* inst, int samples, int s, int ld, int k) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < samples) {
    km_instance in;
    in.offset = (int64_t)q * s * ld;
    in.n = s;
    in.ld = ld;
    in.k = k;
    in.medoid_offset = q * k;
    inst[q] = in;
  }
}

// CLARA's choice on the device: the sample with the least full-data TD
// (lowest index on ties) gives the medoids; its TD, index and the first
// failing sample status (if any) go to the result record.  One block.
__global__ void k_clara_select(const double* sample_td, int samples, const int32_t* smed, int k,
                               const km_batch_result* bres, int32_t* medoids_out,
                               km_clara_result* out, double* sample_td_out) {
  __shared__ int best;
  if (threadIdx.x == 0) {
    int b = 0, st = 0;
    for (int q = 0; q < samples; ++q) {
      if (sample_td[q] < sample_td[b]) b = q;
      if (st == 0 && bres[q].status != 0) st = bres[q].status;
    }
    best = b;
    km_clara_result r;
    r.td = sample_td[b];
    r.best_sample = b;
    r.status = st;
    *out = r;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) medoids_out[j] = smed[(size_t)best * k + j];
  if (sample_td_out)
    for (int q = threadIdx.x; q < samples; q += blockDim.x) sample_td_out[q] = sample_td[q];
}

// CLARA: medoid j of sample q is position smed[q k + j] of that sample;
// replace it by the point index sample_idx[q s + position].
__global__ void k_clara_map(int32_t* smed, const int32_t* sample_idx, int samples, int k, int s) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < samples * k) smed[e] = sample_idx[(long long)(e / k) * s + smed[e]];
}

// CLARA assignment: every point against the k medoids of each of nq samples
// (FP32 direct differences, lowest slot on ties), sqrt of the least squared
// distance summed per sample in FP64.  The medoid coordinates of all nq
// samples sit in shared memory with rows padded to DP4 float4 (zeros), the
// point in registers (zero-padded the same way).  With labels != NULL (one
// sample) the nearest slot of every point is written as well.
// DP4 = 0: any d, the point read from global memory (rows padded to dp4).
template <int DP4>
__global__ void __launch_bounds__(256) k_clara_assign(const float* X, long long n, int d, int dp4,
                                                      const int32_t* med, int k, int nq,
                                                      double* sample_td, int32_t* labels) {
  extern __shared__ float4 sm4[];  // [nq * k][dp4] medoid rows, then [nq][256] FP64 sums
  if (DP4 > 0) dp4 = DP4;
  double* part = reinterpret_cast<double*>(sm4 + (size_t)nq * k * dp4);
  for (int e = threadIdx.x; e < nq * k * dp4 * 4; e += blockDim.x) {
    const int r = e / (dp4 * 4), t = e % (dp4 * 4);
    reinterpret_cast<float*>(sm4)[e] = (t < d) ? X[(long long)med[r] * d + t] : 0.f;
  }
  for (int q = 0; q < nq; ++q) part[q * 256 + threadIdx.x] = 0.0;
  __syncthreads();
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    constexpr int R = DP4 > 0 ? DP4 : 1;
    float4 x[R];
    const float* xo = X + o * d;
#pragma unroll
    for (int t4 = 0; t4 < DP4; ++t4) {
      const int t = 4 * t4;
      x[t4].x = (t < d) ? xo[t] : 0.f;
      x[t4].y = (t + 1 < d) ? xo[t + 1] : 0.f;
      x[t4].z = (t + 2 < d) ? xo[t + 2] : 0.f;
      x[t4].w = (t + 3 < d) ? xo[t + 3] : 0.f;
    }
    for (int q = 0; q < nq; ++q) {
      const float4* mq = sm4 + (size_t)q * k * dp4;
      float best = __int_as_float(0x7f800000);
      int lab = 0;
      for (int j = 0; j < k; ++j) {
        float s2 = 0.f;
        if (DP4 == 0) {
          const float* mr = reinterpret_cast<const float*>(mq + j * dp4);
          for (int t = 0; t < d; ++t) {
            const float df = xo[t] - mr[t];
            s2 = fmaf(df, df, s2);
          }
        }
#pragma unroll
        for (int t4 = 0; t4 < DP4; ++t4) {
          const float4 m = mq[j * DP4 + t4];
          float df = x[t4].x - m.x;
          s2 = fmaf(df, df, s2);
          df = x[t4].y - m.y;
          s2 = fmaf(df, df, s2);
          df = x[t4].z - m.z;
          s2 = fmaf(df, df, s2);
          df = x[t4].w - m.w;
          s2 = fmaf(df, df, s2);
        }
        if (s2 < best) {
          best = s2;
          lab = j;
        }
      }
      part[q * 256 + threadIdx.x] += (double)sqrtf(best);
      if (labels) labels[o] = lab;
    }
  }
  __syncthreads();
  for (int q = 0; q < nq; ++q) {
    double v = part[q * 256 + threadIdx.x];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) part[q * 256 + threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[threadIdx.x * 256 + 32 * w];
    atomicAdd(&sample_td[threadIdx.x], t);
  }
}

}  // namespace km

// ============================================================== host side
using namespace km;

namespace {

km_status bfail(km_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define BK(call)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return bfail(KM_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                                   \
  } while (0)

template <int WARPS, int STAGES>
cudaError_t launch_batch(const BatchArgs& a, int sms, cudaStream_t s) {
  const size_t sm = sizeof(BatchSmem<WARPS, STAGES>);
  cudaError_t e = cudaFuncSetAttribute(k_batch_pam<WARPS, STAGES>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pam<WARPS, STAGES>,
                                                    WARPS * 32, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > a.count) grid = a.count;
  if (grid < 1) grid = 1;
  k_batch_pam<WARPS, STAGES><<<grid, WARPS * 32, sm, s>>>(a);
  return cudaGetLastError();
}

// geometry: 1 .. kBatchGeometries (KM_BATCH_GEOMETRIES)
cudaError_t launch_batch_geometry(int geometry, const BatchArgs& a, int sms, cudaStream_t s) {
#define KM_BATCH_CASE(G, W, S) \
  if (geometry == G) return launch_batch<W, S>(a, sms, s);
  KM_BATCH_GEOMETRIES(KM_BATCH_CASE)
#undef KM_BATCH_CASE
  return cudaErrorInvalidValue;
}

bool batch_geometry_info(int geometry, int* warps, int* stages) {
#define KM_BATCH_INFO(G, W, S) \
  if (geometry == G) {         \
    *warps = W;                \
    *stages = S;               \
    return true;               \
  }
  KM_BATCH_GEOMETRIES(KM_BATCH_INFO)
#undef KM_BATCH_INFO
  return false;
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

template <int DP4>
cudaError_t launch_assign_t(const float* X, long long n, int d, int dp4, const int32_t* med, int k,
                            int nq, double* td, int32_t* labels, int grid, cudaStream_t s) {
  const size_t sm = 16 * (size_t)nq * k * dp4 + 8 * 256 * (size_t)nq;
  cudaError_t e = cudaFuncSetAttribute(k_clara_assign<DP4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_clara_assign<DP4><<<grid, 256, sm, s>>>(X, n, d, dp4, med, k, nq, td, labels);
  return cudaGetLastError();
}

cudaError_t launch_clara_assign(const float* X, long long n, int d, int dp4, const int32_t* med,
                                int k, int nq, double* td, int32_t* labels, int grid,
                                cudaStream_t s) {
  if (dp4 <= 2) return launch_assign_t<2>(X, n, d, 2, med, k, nq, td, labels, grid, s);
  if (dp4 <= 4) return launch_assign_t<4>(X, n, d, 4, med, k, nq, td, labels, grid, s);
  if (dp4 <= 8) return launch_assign_t<8>(X, n, d, 8, med, k, nq, td, labels, grid, s);
  if (dp4 <= 16) return launch_assign_t<16>(X, n, d, 16, med, k, nq, td, labels, grid, s);
  return launch_assign_t<0>(X, n, d, dp4, med, k, nq, td, labels, grid, s);
}

}  // namespace

extern "C" size_t kmedoids_batched_workspace_size(int32_t count) {
  if (count <= 0) return 0;
  return al256(256) + al256(4 * (size_t)count);
}

namespace {

km_status check_batch_args(const float* arena, const km_instance* inst, int32_t count,
                           int32_t* medoids_out, km_batch_result* results, void* ws) {
  if (!arena || !inst || !medoids_out || !results || !ws) return bfail(KM_E_INVALID, "NULL pointer");
  if (count <= 0 || count > kBatchMaxCount)
    return bfail(KM_E_INVALID, "count must be in [1, %d]", kBatchMaxCount);
  if (reinterpret_cast<uintptr_t>(arena) % 16 || reinterpret_cast<uintptr_t>(ws) % 256)
    return bfail(KM_E_INVALID, "arena must be 16-byte and ws 256-byte aligned");
  return KM_OK;
}

km_status batch_options(const km_options* opts, km_options* o, int* geometry) {
  km_default_options(o);
  if (opts) *o = *opts;
  if (o->variant != KM_FASTPAM1 && o->variant != KM_FASTERPAM)
    return bfail(KM_E_UNSUPPORTED, "the batched form runs FastPAM1 or FasterPAM (variant %d)",
                 o->variant);
  if (o->tune < 0 || o->tune > kBatchGeometries)
    return bfail(KM_E_INVALID, "batched tune must be 0 .. %d (kmedoids_batched_autotune picks one)",
                 kBatchGeometries);
  *geometry = o->tune == 0 ? 1 : o->tune;
  return KM_OK;
}

// Enqueues the ordering kernel and the persistent PAM kernel over both
// instance tables of `a` (device work only).
km_status enqueue_batch(BatchArgs& a, unsigned* queue, int32_t* order, const km_options& o,
                        int geometry, bool start_given, cudaStream_t s) {
  BK(cudaMemsetAsync(queue, 0, 256, s));
  k_batch_order<<<(a.count + 255) / 256, 256, 0, s>>>(a.inst, a.count_a, a.inst2, a.count, order);
  BK(cudaGetLastError());
  a.order = order;
  a.queue = queue;
  a.max_iter = o.max_iter > 0 ? o.max_iter : 10000;
  a.tol = o.tol;
  a.start_given = start_given ? 1 : 0;
  a.eager = (o.variant == KM_FASTERPAM) ? 1 : 0;
  BK(launch_batch_geometry(geometry, a, device_sm_count(), s));
  return KM_OK;
}

BatchArgs batch_args(const float* arena, const km_instance* inst, int32_t count,
                     int32_t* medoids, km_batch_result* results) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.arena = arena;
  a.inst = inst;
  a.count = count;
  a.count_a = count;
  a.medoids = medoids;
  a.out = results;
  return a;
}

}  // namespace

static km_status batched_impl(bool start_given, const float* arena, const km_instance* inst,
                              int32_t count, int32_t* medoids_out, km_batch_result* results,
                              const km_options* opts, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nv(start_given ? "kmedoids_swap_batched" : "kmedoids_run_batched");
  set_last_error("");
  km_status r = check_batch_args(arena, inst, count, medoids_out, results, ws);
  if (r != KM_OK) return r;
  if (ws_bytes < kmedoids_batched_workspace_size(count))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  km_options o;
  int geometry = 1;
  r = batch_options(opts, &o, &geometry);
  if (r != KM_OK) return r;
  unsigned char* w = static_cast<unsigned char*>(ws);
  BatchArgs a = batch_args(arena, inst, count, medoids_out, results);
  return enqueue_batch(a, reinterpret_cast<unsigned*>(w), reinterpret_cast<int32_t*>(w + al256(256)),
                       o, geometry, start_given, static_cast<cudaStream_t>(stream));
}

extern "C" km_status kmedoids_run_batched(const float* arena, const km_instance* inst,
                                          int32_t count, int32_t* medoids_out,
                                          km_batch_result* results, const km_options* opts,
                                          void* ws, size_t ws_bytes, void* stream) {
  return batched_impl(false, arena, inst, count, medoids_out, results, opts, ws, ws_bytes, stream);
}

extern "C" km_status kmedoids_swap_batched(const float* arena, const km_instance* inst,
                                           int32_t count, int32_t* medoids_inout,
                                           km_batch_result* results, const km_options* opts,
                                           void* ws, size_t ws_bytes, void* stream) {
  return batched_impl(true, arena, inst, count, medoids_inout, results, opts, ws, ws_bytes,
                      stream);
}

extern "C" int32_t kmedoids_batched_geometry_info(int32_t geometry, int32_t* warps,
                                                  int32_t* stages) {
  int w = 0, st = 0;
  if (!batch_geometry_info(geometry, &w, &st)) return -1;
  if (warps) *warps = w;
  if (stages) *stages = st;
  return 0;
}

// ------------------------------------------------------------- autotuner
// Measured choice of the persistent kernel's geometry for a batch, cached
// per (device, variant, instance-size histogram): counts of instances per
// (floor(log2 n), floor(log2 k)) bucket.
namespace {
std::mutex g_btune_mu;
std::map<std::vector<long long>, int> g_btune;
}  // namespace

extern "C" km_status kmedoids_batched_autotune(const float* arena, const km_instance* inst,
                                               int32_t count, int32_t* medoids_out,
                                               km_batch_result* results, const km_options* opts,
                                               void* ws, size_t ws_bytes, void* stream,
                                               int32_t* geometry_out, double* ms_out) {
  NvtxRange nv("kmedoids_batched_autotune");
  set_last_error("");
  km_status r = check_batch_args(arena, inst, count, medoids_out, results, ws);
  if (r != KM_OK) return r;
  if (!geometry_out) return bfail(KM_E_INVALID, "geometry_out is NULL");
  if (ws_bytes < kmedoids_batched_workspace_size(count))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  km_options o;
  int geometry = 1;
  r = batch_options(opts, &o, &geometry);
  if (r != KM_OK) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<km_instance> hi((size_t)count);
  BK(cudaMemcpyAsync(hi.data(), inst, sizeof(km_instance) * (size_t)count,
                     cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  int dev = 0;
  BK(cudaGetDevice(&dev));
  std::vector<long long> key = {dev, o.variant};
  std::map<std::pair<int, int>, long long> hist;
  for (const km_instance& in : hi) {
    const int ln = in.n > 0 ? 31 - __builtin_clz((unsigned)in.n) : -1;
    const int lk = in.k > 0 ? 31 - __builtin_clz((unsigned)in.k) : -1;
    hist[{ln, lk}] += 1;
  }
  for (auto& e : hist) {
    key.push_back(e.first.first);
    key.push_back(e.first.second);
    key.push_back(e.second);
  }
  if (!ms_out) {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    auto it = g_btune.find(key);
    if (it != g_btune.end()) {
      *geometry_out = it->second;
      return KM_OK;
    }
  }
  unsigned char* w = static_cast<unsigned char*>(ws);
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  int best = 1;
  double best_ms = 1e300;
  for (int g = 1; g <= kBatchGeometries; ++g) {
    double ms_g = -1.0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      BatchArgs a = batch_args(arena, inst, count, medoids_out, results);
      BK(cudaEventRecord(e0, s));
      r = enqueue_batch(a, reinterpret_cast<unsigned*>(w), reinterpret_cast<int32_t*>(w + al256(256)),
                        o, g, false, s);
      if (r != KM_OK) break;
      BK(cudaEventRecord(e1, s));
      BK(cudaStreamSynchronize(s));
      float ms = 0.f;
      BK(cudaEventElapsedTime(&ms, e0, e1));
      ms_g = ms;
    }
    if (r != KM_OK) {
      r = KM_OK;  // a geometry that does not launch here is skipped
      set_last_error("");
      ms_g = -1.0;
    }
    if (ms_out) ms_out[g - 1] = ms_g;
    if (ms_g >= 0.0 && ms_g < best_ms) {
      best_ms = ms_g;
      best = g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms >= 1e300) return bfail(KM_E_CUDA, "no geometry of the batched kernel launched");
  {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune[key] = best;
  }
  *geometry_out = best;
  return KM_OK;
}

extern "C" km_status kmedoids_batched_distances(const float* points, int32_t dim,
                                                const int64_t* point_offsets,
                                                const km_instance* inst, int32_t count,
                                                float* arena, void* stream) {
  set_last_error("");
  if (!points || !point_offsets || !inst || !arena || count <= 0 || dim <= 0)
    return bfail(KM_E_INVALID, "invalid arguments");
  if (count > kBatchMaxCount || dim > kDistMaxDim)
    return bfail(KM_E_UNSUPPORTED, "need count <= %d and dim <= %d", kBatchMaxCount, kDistMaxDim);
  DistArgs a;
  memset(&a, 0, sizeof(a));
  a.P = points;
  a.dim = dim;
  a.point_off = reinterpret_cast<const long long*>(point_offsets);
  a.inst = inst;
  a.D = arena;
  a.count = count;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid(64, count);
  const size_t sm = dist_smem(dim);
  BK(cudaFuncSetAttribute(k_batch_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_batch_dist<<<grid, 256, sm, s>>>(a);
  BK(cudaGetLastError());
  BK(cudaStreamSynchronize(s));
  return KM_OK;
}

// ----------------------------------------------------------------- CLARA
namespace {

// Workspace of the CLARA pipeline: the batch queue and processing order
// (count_a batch instances + the samples), the samples' descriptors,
// results and medoids, the per-sample TDs (+ one scratch slot) and the
// sample matrices.
struct ClaraWs {
  size_t queue, order, inst, bres, smed, std_, arena, total;
};

ClaraWs clara_ws(int count_a, int k, int samples, int sample_size) {
  const int ld = (sample_size + 3) / 4 * 4;
  ClaraWs L;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t r = off;
    off += al256(b);
    return r;
  };
  L.queue = take(256);
  L.order = take(4 * ((size_t)count_a + samples));
  L.inst = take(sizeof(km_instance) * (size_t)samples);
  L.bres = take(sizeof(km_batch_result) * (size_t)samples);
  L.smed = take(4 * (size_t)samples * k);
  L.std_ = take(8 * ((size_t)samples + 1));
  L.arena = take(4 * (size_t)samples * sample_size * ld);
  L.total = off;
  return L;
}

km_status check_clara_args(const float* X, int64_t n, int32_t d, int32_t k, int32_t samples,
                           int32_t sample_size, const int32_t* sample_idx, int32_t* medoids_out,
                           void* ws) {
  if (!X || !sample_idx || !medoids_out || !ws) return bfail(KM_E_INVALID, "NULL pointer");
  if (n <= 0 || d <= 0 || d > kDistMaxDim || k <= 0 || samples <= 0 || samples > kBatchMaxCount ||
      sample_size < k || sample_size > n || sample_size > kBatchMaxN || k > kBatchMaxK)
    return bfail(KM_E_INVALID, "need 1 <= k <= sample_size <= min(n, %d), k <= %d, "
                 "1 <= samples <= %d, d <= %d", kBatchMaxN, kBatchMaxK, kBatchMaxCount, kDistMaxDim);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return bfail(KM_E_INVALID, "ws must be 256-byte aligned");
  const int dp4 = (d + 3) / 4;
  if (16 * (size_t)k * dp4 + 8 * 256 > 200 * 1024)
    return bfail(KM_E_UNSUPPORTED, "k * d too large for the assignment kernel");
  return KM_OK;
}

// The whole CLARA method, and optionally a batch of instances, as device
// work on one stream: sample matrices, one persistent PAM launch over the
// batch and the samples, medoid positions -> point indices, the full-data
// assignment of every sample, the choice of the best sample and the labels
// of its medoids.  Nothing is read back, so the sequence can be captured in
// a CUDA graph.
km_status enqueue_clara(const float* arena, const km_instance* inst, int32_t count,
                        int32_t* medoids_out, km_batch_result* results, const float* X, int64_t n,
                        int32_t d, int32_t k, int32_t samples, int32_t sample_size,
                        const int32_t* sample_idx, int32_t* clara_medoids, int32_t* labels,
                        double* sample_td_out, km_clara_result* clara_res, const km_options& o,
                        int geometry, unsigned char* w, cudaStream_t s, int64_t* launches) {
  const ClaraWs L = clara_ws(count, k, samples, sample_size);
  const int ld = (sample_size + 3) / 4 * 4;
  km_instance* sinst = reinterpret_cast<km_instance*>(w + L.inst);
  km_batch_result* bres = reinterpret_cast<km_batch_result*>(w + L.bres);
  int32_t* smed = reinterpret_cast<int32_t*>(w + L.smed);
  double* std_ = reinterpret_cast<double*>(w + L.std_);
  float* sarena = reinterpret_cast<float*>(w + L.arena);
  k_clara_inst<<<(samples + 255) / 256, 256, 0, s>>>(sinst, samples, sample_size, ld, k);
  BK(cudaGetLastError());
  DistArgs da;
  memset(&da, 0, sizeof(da));
  da.P = X;
  da.dim = d;
  da.idx = sample_idx;
  da.s = sample_size;
  da.inst = sinst;
  da.D = sarena;
  da.count = samples;
  const size_t dsm = dist_smem(d);
  BK(cudaFuncSetAttribute(k_batch_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
  k_batch_dist<<<dim3(64, samples), 256, dsm, s>>>(da);
  BK(cudaGetLastError());
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.arena = arena;
  a.inst = inst;
  a.count_a = count;
  a.medoids = medoids_out;
  a.out = results;
  a.arena2 = sarena;
  a.inst2 = sinst;
  a.medoids2 = smed;
  a.out2 = bres;
  a.count = count + samples;
  km_options ob = o;
  ob.variant = KM_FASTPAM1;  // CLARA's inner method is BUILD + FastPAM1 (FastCLARA)
  if (count > 0 && o.variant == KM_FASTERPAM) {
    // the batch runs FasterPAM: a launch of its own, the samples FastPAM1
    BatchArgs ab = a;
    ab.count = count;
    km_status r = enqueue_batch(ab, reinterpret_cast<unsigned*>(w + L.queue),
                                reinterpret_cast<int32_t*>(w + L.order), o, geometry, false, s);
    if (r != KM_OK) return r;
    a.inst = sinst;
    a.arena = sarena;
    a.medoids = smed;
    a.out = bres;
    a.count_a = samples;
    a.count = samples;
    *launches += 2;
  }
  km_status r = enqueue_batch(a, reinterpret_cast<unsigned*>(w + L.queue),
                              reinterpret_cast<int32_t*>(w + L.order), ob, geometry, false, s);
  if (r != KM_OK) return r;
  k_clara_map<<<(samples * k + 255) / 256, 256, 0, s>>>(smed, sample_idx, samples, k, sample_size);
  BK(cudaGetLastError());
  BK(cudaMemsetAsync(std_, 0, 8 * ((size_t)samples + 1), s));
  const int dp4 = (d + 3) / 4;
  const size_t per_sample = 16 * (size_t)k * dp4 + 8 * 256;
  const size_t smem_cap = 200 * 1024;
  const int group = (int)std::min<size_t>((size_t)samples, smem_cap / per_sample);
  const int agrid = device_sm_count() * 8;
  *launches += 5;  // descriptors, distances, order, PAM, medoid map
  for (int q0 = 0; q0 < samples; q0 += group) {
    const int nq = std::min(group, samples - q0);
    BK(launch_clara_assign(X, n, d, dp4, smed + (size_t)q0 * k, k, nq, std_ + q0, nullptr, agrid, s));
    ++*launches;
  }
  k_clara_select<<<1, 256, 0, s>>>(std_, samples, smed, k, bres, clara_medoids, clara_res,
                                   sample_td_out);
  BK(cudaGetLastError());
  ++*launches;
  if (labels) {
    // labels of the chosen medoids; the TD this pass adds lands in the scratch slot
    BK(launch_clara_assign(X, n, d, dp4, clara_medoids, k, 1, std_ + samples, labels, agrid, s));
    ++*launches;
  }
  return KM_OK;
}

}  // namespace

extern "C" size_t kmedoids_clara_workspace_size(int32_t k, int32_t samples, int32_t sample_size) {
  if (k <= 0 || samples <= 0 || sample_size < k) return 0;
  return clara_ws(0, k, samples, sample_size).total + al256(sizeof(km_clara_result));
}

extern "C" size_t kmedoids_batched_clara_workspace_size(int32_t count, int32_t k, int32_t samples,
                                                        int32_t sample_size) {
  if (count < 0 || k <= 0 || samples <= 0 || sample_size < k) return 0;
  return clara_ws(count, k, samples, sample_size).total;
}

extern "C" km_status kmedoids_clara(const float* X, int64_t n, int32_t d, int32_t k,
                                    int32_t samples, int32_t sample_size,
                                    const int32_t* sample_idx, int32_t* medoids_out,
                                    int32_t* labels_out, double* sample_td_host,
                                    km_result* res, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_clara");
  set_last_error("");
  km_status r = check_clara_args(X, n, d, k, samples, sample_size, sample_idx, medoids_out, ws);
  if (r != KM_OK) return r;
  if (ws_bytes < kmedoids_clara_workspace_size(k, samples, sample_size))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  const ClaraWs L = clara_ws(0, k, samples, sample_size);
  km_clara_result* cres = reinterpret_cast<km_clara_result*>(w + L.total);
  km_options o;
  km_default_options(&o);
  int64_t launches = 0;
  r = enqueue_clara(nullptr, nullptr, 0, nullptr, nullptr, X, n, d, k, samples, sample_size,
                    sample_idx, medoids_out, labels_out, nullptr, cres, o, 1, w, s, &launches);
  if (r != KM_OK) return r;
  km_clara_result hres;
  std::vector<double> tds((size_t)samples);
  BK(cudaMemcpyAsync(&hres, cres, sizeof(hres), cudaMemcpyDeviceToHost, s));
  BK(cudaMemcpyAsync(tds.data(), w + L.std_, 8 * (size_t)samples, cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  if (sample_td_host)
    for (int q = 0; q < samples; ++q) sample_td_host[q] = tds[q];
  if (res) {
    memset(res, 0, sizeof(*res));
    res->td = hres.td;
    res->best_sample = hres.best_sample;
    res->status = hres.status;
    res->kernel_launches = launches;
  }
  if (hres.status != 0) return bfail((km_status)hres.status, "a CLARA sample failed (status %d)",
                                     hres.status);
  return KM_OK;
}

extern "C" km_status kmedoids_run_batched_clara(
    const float* arena, const km_instance* inst, int32_t count, int32_t* medoids_out,
    km_batch_result* results, const float* X, int64_t n, int32_t d, int32_t k, int32_t samples,
    int32_t sample_size, const int32_t* sample_idx, int32_t* clara_medoids_out,
    int32_t* clara_labels_out, double* sample_td, km_clara_result* clara_result,
    const km_options* opts, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_run_batched_clara");
  set_last_error("");
  km_status r;
  if (count > 0) {
    r = check_batch_args(arena, inst, count, medoids_out, results, ws);
    if (r != KM_OK) return r;
  } else if (count < 0) {
    return bfail(KM_E_INVALID, "count must be >= 0");
  }
  r = check_clara_args(X, n, d, k, samples, sample_size, sample_idx, clara_medoids_out, ws);
  if (r != KM_OK) return r;
  if (!clara_result) return bfail(KM_E_INVALID, "clara_result is NULL");
  if (count + (int64_t)samples > kBatchMaxCount)
    return bfail(KM_E_INVALID, "count + samples must be <= %d", kBatchMaxCount);
  if (ws_bytes < kmedoids_batched_clara_workspace_size(count, k, samples, sample_size))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  km_options o;
  int geometry = 1;
  r = batch_options(opts, &o, &geometry);
  if (r != KM_OK) return r;
  int64_t launches = 0;
  return enqueue_clara(count > 0 ? arena : nullptr, count > 0 ? inst : nullptr, count,
                       medoids_out, results, X, n, d, k, samples, sample_size, sample_idx,
                       clara_medoids_out, clara_labels_out, sample_td, clara_result, o, geometry,
                       static_cast<unsigned char*>(ws), static_cast<cudaStream_t>(stream),
                       &launches);
}

// km_batched.cu -- many independent PAM instances in one persistent launch,
// and CLARA (Sec. 2.2; FastCLARA, Sec. 3.3) on top of it.
//
// k_batch_pam: each CTA takes instances from an atomic queue (the host
// orders them largest first) and runs the whole method on one instance:
// BUILD (Alg. 1), the exact per-point cache, and FastPAM1 SWAP (Alg. 3,
// Eq. (7)) to convergence, with every per-point quantity in shared memory
// and one warp per candidate row.  Float sums of the SWAP pass use the same
// exact 64-bit fixed point as the single-instance kernels (scale from the
// instance's largest entry, found during BUILD step 0).  Instances need
// n <= 4096 and k <= 128.
//
// CLARA: the caller passes the sample indices (drawn by its own generator);
// the sample matrices are built with the FP64 recipe below, solved as extra
// instances of k_batch_pam, then every point of the full data set is
// assigned to each sample's medoids (FP32 direct differences, FP64 TD sum)
// and the sample with the least TD wins (lowest index on ties).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"

namespace km {

constexpr int kBatchMaxN = 4096;
constexpr int kBatchMaxK = 128;

struct BatchArgs {
  const float* arena;
  const km_instance* inst;
  int count;
  const int32_t* order;      // instance processing order (largest first)
  int32_t* medoids;          // concatenated, at inst[i].medoid_offset
  km_batch_result* out;
  unsigned* queue;           // next position in order
  int* error;
  int max_iter;
  double tol;
};

// Euclidean matrix of m points (FP64 differences, one rounding to FP32):
// instance/sample q has points P[idx[q][i]] (idx may be NULL: consecutive
// points from point_off[q]) and writes rows of ld elements at D + d_off[q].
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

__global__ void k_batch_dist(const DistArgs a) {
  // grid.y = instance, grid.x x block = rows; one thread per row entry
  const int q = blockIdx.y;
  if (q >= a.count) return;
  const km_instance in = a.inst[q];
  float* D = a.D + in.offset;
  const int m = in.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * in.ld;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / in.ld), j = (int)(e % in.ld);
    float v = 0.f;
    if (j < m) {
      const long long pi = a.idx ? a.idx[(long long)q * a.s + i] : a.point_off[q] + i;
      const long long pj = a.idx ? a.idx[(long long)q * a.s + j] : a.point_off[q] + j;
      const float* xi = a.P + pi * a.dim;
      const float* xj = a.P + pj * a.dim;
      double sq = 0.0;
      for (int t = 0; t < a.dim; ++t) {
        const double df = (double)xi[t] - (double)xj[t];
        sq += df * df;
      }
      v = (float)sqrt(sq);
    }
    D[(size_t)i * in.ld + j] = v;
  }
}

template <int WARPS>
struct BatchSmem {
  float dn[kBatchMaxN];
  float ds[kBatchMaxN];
  uint8_t near[kBatchMaxN];
  uint8_t sec[kBatchMaxN];
  uint8_t is_med[kBatchMaxN];
  int32_t med[kBatchMaxK];
  long long rl[kBatchMaxK];
  long long acc[WARPS][kBatchMaxK + 1];
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

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_batch_pam(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<WARPS>& S = *reinterpret_cast<BatchSmem<WARPS>*>(smem_raw);
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
    const km_instance in = a.inst[q];
    const int n = in.n, k = in.k, ld = in.ld;
    const float* D = a.arena + in.offset;
    km_batch_result res;
    res.td = 0.0;
    res.iterations = 0;
    res.swaps = 0;
    res.status = 0;
    res.pad = 0;
    if (n < 1 || n > kBatchMaxN || k < 1 || k > kBatchMaxK || k > n || ld < n || (ld & 3)) {
      if (tid == 0) {
        res.status = KM_E_INVALID;
        a.out[q] = res;
      }
      __syncthreads();
      continue;
    }
    for (int o = tid; o < n; o += NT) S.is_med[o] = 0;
    __syncthreads();

    // ------------------------------------------------------------- BUILD
    unsigned mloc = 0;
    for (int step = 0; step < k; ++step) {
      double bd = 1e300;
      int bc = INT_MAX;
      for (int c = warp; c < n; c += WARPS) {
        if (S.is_med[c]) continue;
        const float* row = D + (size_t)c * ld;
        float hs = 0.f, hc = 0.f;
        for (int o = lane * 4; o < n; o += 128) {
          const float4 v = *reinterpret_cast<const float4*>(row + o);
          const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (o + t < n) {
              float x;
              if (step == 0) {
                x = e[t];
                mloc = max(mloc, __float_as_uint(e[t]) & 0x7fffffffu);
              } else {
                x = (e[t] < S.dn[o + t]) ? e[t] - S.dn[o + t] : 0.f;
              }
              kahan_add(hs, hc, x);
            }
          }
        }
        const double g = warp_sum_pair(hs, -hc);
        if (g < bd) {  // rows visited in ascending order: keeps the lowest c
          bd = g;
          bc = c;
        }
      }
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

    // --------------------------------------------- cache, removal loss, TD
    auto cache_all = [&]() {
      for (int i = tid; i < k; i += NT) S.rl[i] = 0;
      __syncthreads();
      for (int o = tid; o < n; o += NT) {
        int n1 = -1, n2 = -1;
        float d1 = 0.f, d2 = 0.f;
        for (int j = 0; j < k; ++j) {
          const float v = D[(size_t)S.med[j] * ld + o];
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
        S.near[o] = (uint8_t)n1;
        S.sec[o] = (uint8_t)(n2 < 0 ? 0 : n2);
        S.dn[o] = d1;
        S.ds[o] = (n2 < 0) ? __int_as_float(0x7f800000) : d2;
        if (n2 >= 0) atomic_add_acc(&S.rl[n1], fx_of(d2, f) - fx_of(d1, f));
      }
      __syncthreads();
    };

    if (k < n) {
      cache_all();
      int it = 0;
      bool conv = false;
      while (it < a.max_iter) {
        // ----------------------------------------------- SWAP evaluation
        long long wbest = LLONG_MAX;
        int wslot = INT_MAX, wcand = INT_MAX;
        if (k >= 2) {
          for (int c = warp; c < n; c += WARPS) {
            if (S.is_med[c]) continue;
            long long* ar = S.acc[warp];
            for (int i = lane; i <= k; i += 32) ar[i] = 0;
            __syncwarp();
            const float* row = D + (size_t)c * ld;
            for (int o = lane * 4; o < n; o += 128) {
              const float4 v = *reinterpret_cast<const float4*>(row + o);
              const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const int p = o + t;
                if (p < n && e[t] < S.ds[p]) {
                  const float dnp = S.dn[p], dsp = S.ds[p];
                  const int sl = S.near[p];
                  const long long xd = fx_of(e[t], f), xs = fx_of(dsp, f);
                  if (e[t] < dnp) {
                    const long long xn = fx_of(dnp, f);
                    atomic_add_acc(&ar[k], xd - xn);
                    atomic_add_acc(&ar[sl], xn - xs);
                  } else {
                    atomic_add_acc(&ar[sl], xd - xs);
                  }
                }
              }
            }
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
            const long long tot = bv + ar[k];
            if (tot < wbest || (tot == wbest && (bi < wslot || (bi == wslot && c < wcand)))) {
              wbest = tot;
              wslot = bi;
              wcand = c;
            }
            __syncwarp();
          }
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
      a.out[q] = res;
    }
    for (int j = tid; j < k; j += NT) a.medoids[in.medoid_offset + j] = S.med[j];
    __syncthreads();
  }
}

// CLARA assignment: for each point and each sample, the nearest of the
// sample's k medoids (FP32 direct differences), summed per sample in FP64.
__global__ void __launch_bounds__(256) k_clara_assign(const float* X, long long n, int d,
                                                      const int32_t* med, int k, int samples,
                                                      double* sample_td) {
  extern __shared__ float sm[];  // medoid coordinates of one sample, k x d
  __shared__ double red[8];
  for (int q = 0; q < samples; ++q) {
    for (int e = threadIdx.x; e < k * d; e += blockDim.x)
      sm[e] = X[(long long)med[q * k + e / d] * d + e % d];
    __syncthreads();
    double part = 0.0;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
         o += (long long)gridDim.x * blockDim.x) {
      const float* xo = X + o * d;
      float best = __int_as_float(0x7f800000);
      for (int j = 0; j < k; ++j) {
        float s2 = 0.f;
        for (int t = 0; t < d; ++t) {
          const float df = xo[t] - sm[j * d + t];
          s2 = fmaf(df, df, s2);
        }
        best = fminf(best, s2);
      }
      part += (double)sqrtf(best);
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(&sample_td[q], t);
    }
    __syncthreads();
  }
}

// Labels of every point for the chosen medoids (lowest slot on ties).
__global__ void k_clara_labels(const float* X, long long n, int d, const int32_t* med, int k,
                               int32_t* labels) {
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    const float* xo = X + o * d;
    float best = 0.f;
    int lab = -1;
    for (int j = 0; j < k; ++j) {
      const float* xm = X + (long long)med[j] * d;
      float s2 = 0.f;
      for (int t = 0; t < d; ++t) {
        const float df = xo[t] - xm[t];
        s2 = fmaf(df, df, s2);
      }
      if (lab < 0 || s2 < best) {
        best = s2;
        lab = j;
      }
    }
    labels[o] = lab;
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

template <int WARPS>
cudaError_t launch_batch(const BatchArgs& a, int sms, cudaStream_t s) {
  const size_t sm = sizeof(BatchSmem<WARPS>);
  cudaError_t e = cudaFuncSetAttribute(k_batch_pam<WARPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pam<WARPS>, WARPS * 32, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > a.count) grid = a.count;
  if (grid < 1) grid = 1;
  k_batch_pam<WARPS><<<grid, WARPS * 32, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_cfg(int cfg, const BatchArgs& a, int sms, cudaStream_t s) {
  return cfg == 0 ? launch_batch<8>(a, sms, s) : launch_batch<16>(a, sms, s);
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" size_t kmedoids_batched_workspace_size(int32_t count) {
  if (count <= 0) return 0;
  return al256(256) + al256(4 * (size_t)count);
}

extern "C" km_status kmedoids_run_batched(const float* arena, const km_instance* inst,
                                          int32_t count, int32_t* medoids_out,
                                          km_batch_result* results, const km_options* opts,
                                          void* ws, size_t ws_bytes, void* stream) {
  set_last_error("");
  if (!arena || !inst || !medoids_out || !results || !ws) return bfail(KM_E_INVALID, "NULL pointer");
  if (count <= 0) return bfail(KM_E_INVALID, "count must be positive");
  if (reinterpret_cast<uintptr_t>(arena) % 16 || reinterpret_cast<uintptr_t>(ws) % 256)
    return bfail(KM_E_INVALID, "arena must be 16-byte and ws 256-byte aligned");
  if (ws_bytes < kmedoids_batched_workspace_size(count))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  km_options def;
  km_default_options(&def);
  const km_options o = opts ? *opts : def;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // order instances by work (n^2 (k + 1)), largest first
  std::vector<km_instance> h((size_t)count);
  BK(cudaMemcpyAsync(h.data(), inst, sizeof(km_instance) * count, cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  std::vector<int32_t> ord((size_t)count);
  for (int i = 0; i < count; ++i) {
    ord[i] = i;
    if (h[i].n < 1 || h[i].n > kBatchMaxN || h[i].k < 1 || h[i].k > kBatchMaxK || h[i].k > h[i].n ||
        h[i].ld < h[i].n || h[i].ld % 4 || h[i].offset % 4 || h[i].offset < 0)
      return bfail(KM_E_INVALID, "instance %d: need 1 <= k <= n <= %d, k <= %d, ld >= n, ld and "
                   "offset multiples of 4", i, kBatchMaxN, kBatchMaxK);
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const double wx = (double)h[x].n * h[x].n * (h[x].k + 1), wy = (double)h[y].n * h[y].n * (h[y].k + 1);
    return wx > wy;
  });
  unsigned char* w = static_cast<unsigned char*>(ws);
  unsigned* queue = reinterpret_cast<unsigned*>(w);
  int32_t* order = reinterpret_cast<int32_t*>(w + al256(256));
  BK(cudaMemsetAsync(queue, 0, 256, s));
  BK(cudaMemcpyAsync(order, ord.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, s));
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.arena = arena;
  a.inst = inst;
  a.count = count;
  a.order = order;
  a.medoids = medoids_out;
  a.out = results;
  a.queue = queue;
  a.max_iter = o.max_iter > 0 ? o.max_iter : 10000;
  a.tol = o.tol;
  const int sms = device_sm_count();
  // tune: 0 automatic (16 warps per CTA), 1 = 8 warps, 2 = 16 warps
  const int cfg = (o.tune == 1) ? 0 : 1;
  BK(launch_batch_cfg(cfg, a, sms, s));
  BK(cudaStreamSynchronize(s));
  return KM_OK;
}

extern "C" km_status kmedoids_batched_distances(const float* points, int32_t dim,
                                                const int64_t* point_offsets,
                                                const km_instance* inst, int32_t count,
                                                float* arena, void* stream) {
  set_last_error("");
  if (!points || !point_offsets || !inst || !arena || count <= 0 || dim <= 0)
    return bfail(KM_E_INVALID, "invalid arguments");
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
  k_batch_dist<<<grid, 256, 0, s>>>(a);
  BK(cudaGetLastError());
  BK(cudaStreamSynchronize(s));
  return KM_OK;
}

extern "C" size_t kmedoids_clara_workspace_size(int32_t k, int32_t samples, int32_t sample_size) {
  if (k <= 0 || samples <= 0 || sample_size < k) return 0;
  const int ld = (sample_size + 3) / 4 * 4;
  return al256(kmedoids_batched_workspace_size(samples)) +
         al256(sizeof(km_instance) * (size_t)samples) +
         al256(sizeof(km_batch_result) * (size_t)samples) + al256(4 * (size_t)samples * k) +
         al256(8 * (size_t)samples) + al256(4 * (size_t)samples * sample_size * ld);
}

extern "C" km_status kmedoids_clara(const float* X, int64_t n, int32_t d, int32_t k,
                                    int32_t samples, int32_t sample_size,
                                    const int32_t* sample_idx, int32_t* medoids_out,
                                    int32_t* labels_out, double* sample_td_host,
                                    km_result* res, void* ws, size_t ws_bytes, void* stream) {
  set_last_error("");
  if (!X || !sample_idx || !medoids_out || !ws) return bfail(KM_E_INVALID, "NULL pointer");
  if (n <= 0 || d <= 0 || k <= 0 || samples <= 0 || sample_size < k || sample_size > n ||
      sample_size > kBatchMaxN || k > kBatchMaxK)
    return bfail(KM_E_INVALID, "need 1 <= k <= sample_size <= min(n, %d), k <= %d, samples >= 1",
                 kBatchMaxN, kBatchMaxK);
  if (ws_bytes < kmedoids_clara_workspace_size(k, samples, sample_size))
    return bfail(KM_E_WORKSPACE, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ld = (sample_size + 3) / 4 * 4;
  unsigned char* w = static_cast<unsigned char*>(ws);
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* p = w + off;
    off += al256(b);
    return p;
  };
  unsigned char* bws = take(kmedoids_batched_workspace_size(samples));
  km_instance* inst = reinterpret_cast<km_instance*>(take(sizeof(km_instance) * samples));
  km_batch_result* bres = reinterpret_cast<km_batch_result*>(take(sizeof(km_batch_result) * samples));
  int32_t* smed = reinterpret_cast<int32_t*>(take(4 * (size_t)samples * k));
  double* std_ = reinterpret_cast<double*>(take(8 * (size_t)samples));
  float* arena = reinterpret_cast<float*>(take(4 * (size_t)samples * sample_size * ld));
  std::vector<km_instance> hi((size_t)samples);
  for (int q = 0; q < samples; ++q) {
    hi[q].offset = (int64_t)q * sample_size * ld;
    hi[q].n = sample_size;
    hi[q].ld = ld;
    hi[q].k = k;
    hi[q].medoid_offset = q * k;
  }
  BK(cudaMemcpyAsync(inst, hi.data(), sizeof(km_instance) * samples, cudaMemcpyHostToDevice, s));
  DistArgs da;
  memset(&da, 0, sizeof(da));
  da.P = X;
  da.dim = d;
  da.idx = sample_idx;
  da.s = sample_size;
  da.inst = inst;
  da.D = arena;
  da.count = samples;
  k_batch_dist<<<dim3(64, samples), 256, 0, s>>>(da);
  BK(cudaGetLastError());
  km_options o;
  km_default_options(&o);
  km_status r = kmedoids_run_batched(arena, inst, samples, smed, bres, &o, bws,
                                     kmedoids_batched_workspace_size(samples), stream);
  if (r != KM_OK) return r;
  // map sample-local medoids to point indices (device gather on the host path)
  std::vector<int32_t> hm((size_t)samples * k), hs((size_t)samples * sample_size);
  BK(cudaMemcpyAsync(hm.data(), smed, 4 * hm.size(), cudaMemcpyDeviceToHost, s));
  BK(cudaMemcpyAsync(hs.data(), sample_idx, 4 * hs.size(), cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  for (int q = 0; q < samples; ++q)
    for (int j = 0; j < k; ++j) hm[(size_t)q * k + j] = hs[(size_t)q * sample_size + hm[(size_t)q * k + j]];
  BK(cudaMemcpyAsync(smed, hm.data(), 4 * hm.size(), cudaMemcpyHostToDevice, s));
  BK(cudaMemsetAsync(std_, 0, 8 * (size_t)samples, s));
  const size_t sm = 4 * (size_t)k * d;
  if (sm > 200 * 1024) return bfail(KM_E_UNSUPPORTED, "k * d too large for the assignment kernel");
  BK(cudaFuncSetAttribute(k_clara_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int grid = device_sm_count() * 4;
  k_clara_assign<<<grid, 256, sm, s>>>(X, n, d, smed, k, samples, std_);
  BK(cudaGetLastError());
  std::vector<double> tds((size_t)samples);
  BK(cudaMemcpyAsync(tds.data(), std_, 8 * (size_t)samples, cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  int best = 0;
  for (int q = 1; q < samples; ++q)
    if (tds[q] < tds[best]) best = q;
  BK(cudaMemcpyAsync(medoids_out, smed + (size_t)best * k, 4 * (size_t)k, cudaMemcpyDeviceToDevice, s));
  if (labels_out) {
    k_clara_labels<<<device_sm_count() * 4, 256, 0, s>>>(X, n, d, smed + (size_t)best * k, k,
                                                         labels_out);
    BK(cudaGetLastError());
  }
  BK(cudaStreamSynchronize(s));
  if (sample_td_host)
    for (int q = 0; q < samples; ++q) sample_td_host[q] = tds[q];
  if (res) {
    memset(res, 0, sizeof(*res));
    res->td = tds[best];
    res->best_sample = best;
    res->status = KM_OK;
  }
  return KM_OK;
}

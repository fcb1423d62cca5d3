// km_gram.cu -- BF16 feature preparation for the on-the-fly distance form and
// a plain tensor-core Gram product G = X X^T (tcgen05, FP32 accumulation in
// tensor memory).  The Gram entry point exists to validate the MMA operand
// layout, descriptors and TMEM read-back on their own; the fused SWAP and
// BUILD kernels of km_features.cu use the same pieces.
#define KM_SRC_ID 8  // names this file in bounds-check reports
#include <cstdio>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"
#include "km_tc.cuh"

namespace km {

// X (n x d bf16, row-major, row stride ldx elements) -> Xp in the K-major
// core-matrix layout of km_tc.cuh, n_pad = roundup(n, 128) rows, zero rows
// beyond n.  One thread per 16-byte chunk (8 elements) of Xp.
__global__ void k_prearrange(const uint16_t* __restrict__ X, long long ldx, int n, int d,
                             int n_pad, uint16_t* __restrict__ Xp) {
  const long long chunks = (long long)n_pad * (d / 8);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < chunks;
       q += (long long)gridDim.x * blockDim.x) {
    // destination chunk q: group g, k-core kc, row-in-group rr
    const long long per_group = (long long)(d / 8) * 8;
    const long long g = q / per_group;
    const long long rem = q - g * per_group;
    const int kc = (int)(rem / 8), rr = (int)(rem % 8);
    const long long row = g * 8 + rr;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (row < n) v = *reinterpret_cast<const uint4*>(X + row * ldx + kc * 8);
    reinterpret_cast<uint4*>(Xp)[q] = v;
  }
}

// ||x_o||^2 in FP32 from the bf16 values (products are exact in FP32).
__global__ void k_row_norms(const uint16_t* __restrict__ X, long long ldx, int n, int d,
                            int n_pad, float* __restrict__ norms) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_pad) return;
  float s = 0.f;
  if (o < n)
    for (int t = 0; t < d; ++t) {
      const float v = __uint_as_float((uint32_t)X[(long long)o * ldx + t] << 16);
      s = fmaf(v, v, s);
    }
  norms[o] = s;
}

// One 128 x 128 tile of G per CTA (4 warps).  Thread 0 stages both operand
// tiles with 1-D bulk copies and issues the d/16 MMAs; every warp then reads
// its 32 TMEM lanes back.  All waits are bounded; a timeout sets *err.
__global__ void __launch_bounds__(128) k_gram_tile(const uint16_t* __restrict__ Xp, int n, int d,
                                                   float* __restrict__ G, long long ldg,
                                                   int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = blockIdx.y, tj = blockIdx.x;
  const size_t tile_bytes = (size_t)kTileM * d * 2;
  unsigned char* sA = smem;
  unsigned char* sB = smem + tile_bytes;
  if (tid == 0) {
    mbar_init(&bar_load, 1);
    mbar_init(&bar_mma, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, kTileN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  volatile int* ab = &abort_flag;

  if (tid == 0) {
    mbar_arrive_expect_tx(&bar_load, (uint32_t)(2 * tile_bytes));
    bulk_g2s(sA, Xp + (size_t)ti * kTileM * d, (uint32_t)tile_bytes, &bar_load);
    bulk_g2s(sB, Xp + (size_t)tj * kTileN * d, (uint32_t)tile_bytes, &bar_load);
    if (mbar_wait(&bar_load, 0, ab)) {
      tc_fence_after();
      const uint32_t idesc = make_idesc_bf16(kTileM, kTileN);
      const uint32_t lbo = 128, sbo = 16u * (uint32_t)d;
      for (int ks = 0; ks < d / 16; ++ks) {
        const uint64_t a = make_sdesc(smem_u32(sA) + ks * 256, lbo, sbo);
        const uint64_t b = make_sdesc(smem_u32(sB) + ks * 256, lbo, sbo);
        umma_bf16(tbase, a, b, idesc, ks > 0 ? 1u : 0u);
      }
      umma_commit(&bar_mma);
    } else {
      *ab = 1;
      atomicExch(err, kErrTimeout);
    }
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar_mma, 0, ab);
  tc_fence_after();
  if (ok) {
    const int row = ti * kTileM + warp * 32 + lane;
    for (int c0 = 0; c0 < kTileN; c0 += 32) {
      float v[32];
      tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_ld_wait();
      if (row < n)
        for (int c = 0; c < 32; ++c) {
          const int col = tj * kTileN + c0 + c;
          if (col < n) G[(size_t)row * ldg + col] = v[c];
        }
    }
  } else if (tid == 0) {
    atomicExch(err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, kTileN);
}

cudaError_t launch_prearrange(const void* X, long long ldx, int n, int d, int n_pad, void* Xp,
                              cudaStream_t s) {
  const long long chunks = (long long)n_pad * (d / 8);
  int grid = (int)((chunks + 255) / 256);
  if (grid > 65535 * 8) grid = 65535 * 8;
  k_prearrange<<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(X), ldx, n, d, n_pad,
                                    static_cast<uint16_t*>(Xp));
  return cudaGetLastError();
}

cudaError_t launch_row_norms(const void* X, long long ldx, int n, int d, int n_pad, float* norms,
                             cudaStream_t s) {
  k_row_norms<<<(n_pad + 255) / 256, 256, 0, s>>>(static_cast<const uint16_t*>(X), ldx, n, d,
                                                   n_pad, norms);
  return cudaGetLastError();
}

}  // namespace km

using namespace km;

extern "C" km_status kmedoids_gram_bf16(const void* X, int64_t n, int32_t d, int64_t ldx,
                                        float* G, int64_t ldg, void* ws, size_t ws_bytes,
                                        void* stream) {
  char msg[256];
  if (!X || !G || !ws) {
    set_last_error("kmedoids_gram_bf16: NULL pointer");
    return KM_E_INVALID;
  }
  if (n <= 0 || n > (1 << 20) || d <= 0 || d > 256 || d % 16 != 0 || ldx < d || ldx % 8 != 0 ||
      ldg < n) {
    snprintf(msg, sizeof(msg),
             "kmedoids_gram_bf16: need 0 < n <= 2^20, d a multiple of 16 up to 256, ldx >= d "
             "and a multiple of 8, ldg >= n (n=%lld d=%d ldx=%lld ldg=%lld)",
             (long long)n, d, (long long)ldx, (long long)ldg);
    set_last_error(msg);
    return KM_E_INVALID;
  }
  if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(ws) % 256) {
    set_last_error("kmedoids_gram_bf16: X must be 16-byte and ws 256-byte aligned");
    return KM_E_INVALID;
  }
  const int n_pad = (int)((n + kTileM - 1) / kTileM * kTileM);
  const size_t need = (size_t)n_pad * d * 2 + 256;
  if (ws_bytes < need) {
    snprintf(msg, sizeof(msg), "kmedoids_gram_bf16: workspace too small: %zu < %zu", ws_bytes,
             need);
    set_last_error(msg);
    return KM_E_WORKSPACE;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  int* err = reinterpret_cast<int*>(w);
  void* Xp = w + 256;
  cudaError_t e = cudaMemsetAsync(err, 0, 4, s);
  if (e == cudaSuccess) e = launch_prearrange(X, ldx, (int)n, d, n_pad, Xp, s);
  const size_t smem = (size_t)2 * kTileM * d * 2;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    dim3 grid(n_pad / kTileN, n_pad / kTileM);
    k_gram_tile<<<grid, 128, smem, s>>>(static_cast<const uint16_t*>(Xp), (int)n, d, G, ldg, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "kmedoids_gram_bf16: %s", cudaGetErrorString(e));
    set_last_error(msg);
    return KM_E_CUDA;
  }
  if (herr) {
    set_last_error("kmedoids_gram_bf16: a device-side wait timed out");
    return KM_E_TIMEOUT;
  }
  return KM_OK;
}

// km_selftest.cu -- kmedoids_wait_selftest: runs the library's bounded-wait
// routines (mbarrier phase wait, consumer barrier, grid barrier) on a wait
// that can never be satisfied, so that the give-up path -- limit reached,
// KM_E_TIMEOUT recorded in the device state record, kernel returns -- is
// exercised without faulting or hanging the GPU.  Nothing is in flight when
// a wait gives up: no bulk copy, no MMA, no tensor memory.
#define KM_SRC_ID 9  // names this file in bounds-check reports
#include <cstdio>
#include <cstring>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"

namespace km {
namespace {

constexpr long long kSelftestMaxNs = 10000000000ll;  // 10 s

// kind 0: one thread waits for phase 0 of an mbarrier that expects one
//         arrival that never comes.
// kind 1: a consumer barrier of two warps; warp 1 leaves without arriving.
// kind 2: the grid barrier over two CTAs; CTA 1 leaves without arriving.
// kind 3: the bounds-check recorder: the index 5 checked against the bound
//         3 (no memory is accessed with it).
__global__ void k_wait_selftest(KmState* st, int kind) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int never;
  __shared__ int s_ok;
  const unsigned long long lim = wait_limit(st);
  if (kind == 3) {
    if (threadIdx.x == 0) {
      volatile int bad = 5;  // not a constant the compiler could fold
      (void)KM_INB(st, bad, 3);
    }
    return;
  }
  if (kind == 2) {
    if (blockIdx.x != 0) return;
    unsigned epoch = 0;
    (void)grid_barrier(st->bar, epoch, st, &s_ok, lim);  // records the timeout
    return;
  }
  if (threadIdx.x == 0) {
    never = 0;
    mbar_init(&bar, kind == 0 ? 1u : 2u);
    fence_barrier_init();
  }
  __syncthreads();
  if (kind == 0) {
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, &never, lim)) atomicExch(&st->error, kErrTimeout);
    return;
  }
  if (threadIdx.x >= 32) return;  // the warp that never arrives
  uint32_t phase = 0;
  const bool ok = cons_sync(&bar, phase, &never, lim);
  if (!ok && threadIdx.x == 0) atomicExch(&st->error, kErrTimeout);
}

km_status st_fail(km_status s, const char* fmt, long long v) {
  char buf[256];
  snprintf(buf, sizeof(buf), fmt, v);
  set_last_error(buf);
  return s;
}

}  // namespace
}  // namespace km

using namespace km;

extern "C" km_status kmedoids_wait_selftest(int32_t kind, int64_t limit_ns, void* ws,
                                            size_t ws_bytes, void* stream) {
  set_last_error("");
  if (kind < 0 || kind > 3) return st_fail(KM_E_INVALID, "kind must be 0 .. 3 (got %lld)", kind);
  if (limit_ns < 0 || limit_ns > kSelftestMaxNs)
    return st_fail(KM_E_INVALID, "limit_ns must be in 0 .. 1e10 (got %lld)", (long long)limit_ns);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < 512)
    return st_fail(KM_E_INVALID, "ws must be a 256-byte aligned buffer of >= 512 bytes (%lld)",
                   (long long)ws_bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KmState h;
  memset(&h, 0, sizeof(h));
  h.last = -1;
  h.wait_ns = (unsigned long long)limit_ns;
  KmState* st = static_cast<KmState*>(ws);
  cudaError_t e = cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const int grid = (kind == 2) ? 2 : 1;
    const int block = (kind == 1) ? 64 : 32;
    k_wait_selftest<<<grid, block, 0, s>>>(st, kind);
    e = cudaGetLastError();
  }
  KmState r;
  memset(&r, 0, sizeof(r));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, st, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    set_last_error(buf);
    return KM_E_CUDA;
  }
  if (r.error) {
    char buf[256];
    const int code = state_message(r, buf, sizeof(buf));
    set_last_error(buf);
    return (km_status)code;
  }
  return KM_OK;
}

extern "C" int32_t kmedoids_bounds_checked(void) {
#ifdef KM_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

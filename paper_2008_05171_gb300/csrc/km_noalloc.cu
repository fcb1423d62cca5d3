// km_noalloc.cu -- kmedoids_eval_swaps_static: the FastPAM1 evaluation pass
// of kmedoids_eval_swaps for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they evaluate swaps: code running while a memory pool is
// frozen or pinned to a fixed budget, plugins that must not touch the host
// process's allocator, or real-time loops where an allocation could block
// on device synchronisation.  For them this entry point takes its scratch
// from a fixed array in device memory that is part of the loaded library
// image.  Every GPU that loads the library holds this array until the
// process exits.
//
// The scratch array's symbol, used from host code, is only a host-side
// stand-in; its device address is looked up on every call with
// cudaGetSymbolAddress for the current device (it allocates nothing and
// stays right after a cudaDeviceReset reloads the module).
#define KM_SRC_ID 11  // names this file in bounds-check reports
#include <cstdio>
#include <cstring>

#include "../../include/kmedoids.h"
#include "km_internal.h"

namespace {

// Scratch limits of the allocation-free entry point.
constexpr int64_t kStaticMaxN = 32768;
constexpr int32_t kStaticMaxK = 512;
constexpr size_t kStaticBytes = size_t(2) << 20;  // 2 MiB

static __device__ __align__(256) unsigned char km_static_scratch[kStaticBytes];

// Device address of the scratch array on the current device.
cudaError_t scratch_address(void** out) { return cudaGetSymbolAddress(out, km_static_scratch); }

}  // namespace

extern "C" km_status kmedoids_eval_swaps_static(const void* D, int32_t dtype, int64_t n,
                                                int64_t ld, int32_t k, const int32_t* medoids,
                                                double* cand_delta, int32_t* cand_slot,
                                                double* best_delta, int32_t* best_slot,
                                                int32_t* best_cand, void* stream) {
  if (n > kStaticMaxN || k > kStaticMaxK) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "kmedoids_eval_swaps_static: n=%lld, k=%d exceed its fixed scratch "
             "(n <= %lld, k <= %d); use kmedoids_eval_swaps with a workspace",
             (long long)n, k, (long long)kStaticMaxN, kStaticMaxK);
    km::set_last_error(msg);
    return KM_E_UNSUPPORTED;
  }
  const size_t need = kmedoids_workspace_size(n, k, dtype, nullptr);
  if (need == 0)  // invalid sizes: let the regular entry point report them
    return kmedoids_eval_swaps(D, dtype, n, ld, k, medoids, cand_delta, cand_slot, best_delta,
                               best_slot, best_cand, nullptr, 0, stream);
  if (need > kStaticBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "kmedoids_eval_swaps_static: needs %zu bytes of scratch, %zu available", need,
             kStaticBytes);
    km::set_last_error(msg);
    return KM_E_UNSUPPORTED;
  }
  void* ws = nullptr;
  const cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "kmedoids_eval_swaps_static: cudaGetSymbolAddress: %s",
             cudaGetErrorString(e));
    km::set_last_error(msg);
    return KM_E_CUDA;
  }
  // kmedoids_eval_swaps clears every scratch field it relies on (state
  // record, medoid flags, removal-loss and TD buffers) before its kernels
  // read them, so the previous call's leftovers do no harm.
  return kmedoids_eval_swaps(D, dtype, n, ld, k, medoids, cand_delta, cand_slot, best_delta,
                             best_slot, best_cand, ws, kStaticBytes, stream);
}

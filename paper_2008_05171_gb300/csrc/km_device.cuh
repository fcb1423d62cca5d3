// km_device.cuh -- device-side building blocks shared by the kernels of
// libkmedoids: launch geometry, the device state record, reduction keys, and
// thin inline-PTX wrappers for mbarriers and 1-D bulk (TMA) copies.
#pragma once

#include <cstdint>
#include <climits>
#include <cstdio>
#include <cuda_runtime.h>

namespace km {

// ---------------------------------------------------------------- geometry
constexpr int kChunk = 1024;                   // matrix columns per stage
constexpr int kConsWarps = 8;                  // consumer warps per CTA
constexpr int kConsThreads = kConsWarps * 32;  // each owns 4 columns
constexpr int kThreads = kConsThreads + 32;    // + one producer warp
constexpr int kMaxGrid = 1024;                 // workspace bound on CTAs
constexpr int kMaxRows = 16;                   // largest candidate tile
constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // 4 s: the default limit

static_assert(kConsThreads * 4 == kChunk, "4 columns per consumer thread");

// Status codes written by kernels (same values as km_status).
constexpr int kErrTimeout = 5;
constexpr int kErrNumeric = 6;
constexpr int kErrBounds = 8;

// ---------------------------------------------------------- device state
// One record per call, in the workspace.  Kernels read it to pick buffers
// and write the decisions of each pass, so a whole SWAP loop can be enqueued
// without the host looking at intermediate results.
struct KmState {
  int iter;          // evaluation passes completed
  int swaps;         // swaps applied
  int done;          // 1: converged / nothing left to do
  int error;         // km_status of a device-detected failure, 0 if none
  unsigned ticket;   // last-block-done counter of the running kernel
  int rb;            // which removal-loss / TD buffer is current (0/1)
  int accept;        // 1: a swap (best_*) is pending for the apply kernel
  int build_step;    // BUILD steps committed
  double best_d;     // pending / best swap: Delta (float data)
  long long best_i;  // pending / best swap: Delta (integer data)
  int best_slot;
  int best_cand;
  double build_gain_d;      // BUILD: best gain of the current step
  long long build_gain_i;
  int build_cand;
  int ntrace;               // swaps recorded in the trace
  double td_book_d;         // bookkept TD (initial + applied deltas)
  long long td_book_i;
  double build_td_d;        // exact TD after the last BUILD commit
  long long build_td_i;
  long long pos;            // FasterPAM: absolute scan position
  long long last;           // FasterPAM: absolute position of last swap
  int fp2_extra;            // FastPAM2: additional slots queued this pass
  int loop_guard;           // bodies of the SWAP loop graph run so far
  double fp2_dstar;         // FastPAM2: |Delta*| of the pass
  long long fp2_dstar_i;
  unsigned tile_next;       // next candidate tile of the running pass
  unsigned scan_max;        // matrix scan: largest |d| (float bits)
  unsigned scan_bad;        // matrix scan: 1 if an entry is < 0 or not finite
  long long fails;          // FastCLARANS: consecutive failed draws
  long long evaluated;      // FastCLARANS: draws evaluated
  long long win_len;        // FasterPAM / FastCLARANS: next window length
  unsigned bar[2];          // grid barrier of the eager kernel: count, generation
  unsigned check_flags;     // input check: 1 asymmetric, 2 diagonal, 4 value
  unsigned pad1;
  unsigned long long wait_ns;  // limit of every bounded wait (0: kWaitLimitNs)
  long long bad_index;      // bounds-checking build: first index out of range,
  long long bad_bound;      //   the bound it broke,
  int bad_line;             //   the source line of the check (0: none)
  int bad_src;              //   and the translation unit (KM_SRC_ID)
};
static_assert(sizeof(KmState) <= 512, "the workspaces reserve 512 bytes for the state record");

// ------------------------------------------------- bounds-checking build
// Built with -DKM_BOUNDS_CHECK, every index a kernel loads from memory (a
// medoid, a nearest / second slot, a candidate, a list entry, a draw, a
// descriptor offset) is checked against the array it indexes before use.
// An index out of range records KM_E_BOUNDS with the index, its bound and
// the place of the check in the state record, and the access is skipped
// (the kernels then stop at their next check of st->error); nothing traps.
// Without the flag KM_INB is the constant true and costs nothing.
#ifndef KM_SRC_ID
#define KM_SRC_ID 0
#endif
#ifdef KM_BOUNDS_CHECK
static __device__ __noinline__ bool km_index_fault(KmState* st, long long i, long long n,
                                                   int src, int line) {
  if (atomicCAS(&st->bad_line, 0, line) == 0) {
    st->bad_index = i;
    st->bad_bound = n;
    st->bad_src = src;
  }
  atomicCAS(&st->error, 0, kErrBounds);
  return false;
}
#define KM_INB(st, i, n)                                                           \
  ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ||     \
   ::km::km_index_fault((st), (long long)(i), (long long)(n), KM_SRC_ID, __LINE__))
#else
#define KM_INB(st, i, n) true
#endif

// Host: the message of a failure a kernel recorded in a state record (a
// wait that gave up, an index out of range, another status); returns the
// status.
inline int state_message(const KmState& h, char* buf, size_t len) {
  static const char* const src[] = {"?",           "km_stream.cu",   "km_points.cu",
                                    "km_build.cu", "km_eager.cu",    "km_features.cu",
                                    "km_batched.cu", "km_init.cu",   "km_gram.cu",
                                    "km_selftest.cu", "km_api.cu",   "km_noalloc.cu",
                                    "km_upload.cu"};
  if (h.error == kErrTimeout) {
    snprintf(buf, len, "a device wait gave up after its limit of %llu ns",
             h.wait_ns ? h.wait_ns : kWaitLimitNs);
  } else if (h.error == kErrBounds) {
    const int id = (h.bad_src >= 0 && h.bad_src < 13) ? h.bad_src : 0;
    snprintf(buf, len, "index %lld out of range [0, %lld) at %s:%d", h.bad_index, h.bad_bound,
             src[id], h.bad_line);
  } else {
    snprintf(buf, len, "device reported status %d", h.error);
  }
  return h.error;
}

// The limit of the bounded waits of a call (set by the host in the state
// record; 0 selects the default).
__device__ __forceinline__ unsigned long long wait_limit(const KmState* st) {
  const unsigned long long w = st->wait_ns;
  return w ? w : kWaitLimitNs;
}

// Trace record of an applied swap.
struct TraceRec {
  double d;
  long long di;
  int slot;
  int cand;
  long long t_ns;
};

// Reduction key: lexicographic (delta, slot, cand).  For BUILD the slot is
// unused (0) and cand is the point index.
template <class A>
struct Key {
  A d;
  int slot;
  int cand;
};

// Load a key written by another CTA of the running kernel (L2, not L1).
template <class A>
__device__ __forceinline__ Key<A> ld_cg_key(const Key<A>* p) {
  Key<A> r;
  r.d = __ldcg(&p->d);
  r.slot = __ldcg(&p->slot);
  r.cand = __ldcg(&p->cand);
  return r;
}

template <class A>
__device__ __forceinline__ bool key_less(const Key<A>& a, const Key<A>& b) {
  if (a.d != b.d) return a.d < b.d;
  if (a.slot != b.slot) return a.slot < b.slot;
  return a.cand < b.cand;
}

// --------------------------------------------------------- type traits
// SWAP accumulators are 64-bit integers for both data types.  Integer
// distances enter unchanged.  Float distances enter as exact fixed-point
// values floor(x * 2^f), with f chosen per call from the largest matrix
// entry M and n so that every sum the SWAP pass forms (at most 3 n M) fits
// in 62 bits: each term keeps ~60 - log2(n) significant bits relative to M
// and the sums are exact and independent of the summation order.  BUILD
// gains and TD sums use G (FP64 for float data, int64 for integer data).
template <class T>
struct Tr;

// floor(x * 2^f) for a finite x >= 0, computed with integer operations only
// (the FP64 pipe of GB300 is narrow) and without branches.  x < 2^(60 -
// log2(n) - f) by the choice of f, so the left shift stays below 2^62.
__device__ __forceinline__ long long fx_of(float x, int f) {
  const unsigned u = __float_as_uint(x) & 0x7fffffffu;
  const int e = (int)(u >> 23);
  const unsigned m = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int sh = (e ? e : 1) - 150 + f;  // x = m * 2^(sh - f)
  const int l = min(max(sh, 0), 62);
  const int r = min(max(-sh, 0), 63);
  return (long long)(((unsigned long long)m << l) >> r);
}

template <>
struct Tr<float> {
  using A = long long;  // SWAP accumulator (fixed point)
  using G = double;     // BUILD gains, TD
  __device__ __forceinline__ static float low() { return -__int_as_float(0x7f800000); }
  __device__ __forceinline__ static float high() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static double g_high() { return __longlong_as_double(0x7ff0000000000000ll); }
  __device__ __forceinline__ static long long fx(float x, int f) { return fx_of(x, f); }
  __device__ __forceinline__ static double unfx(long long v, int f) { return ldexp((double)v, -f); }
};

template <>
struct Tr<int32_t> {
  using A = long long;
  using G = long long;
  __device__ __forceinline__ static int32_t low() { return INT_MIN; }
  __device__ __forceinline__ static int32_t high() { return INT_MAX; }
  __device__ __forceinline__ static long long g_high() { return LLONG_MAX; }
  __device__ __forceinline__ static long long fx(int32_t x, int) { return (long long)x; }
  __device__ __forceinline__ static double unfx(long long v, int) { return (double)v; }
};

// Value type of a stored matrix element: 16-bit unsigned distances (the
// compressed integer form) are widened to int32, which is exact; int32 and
// float32 elements are used as stored.
template <class E>
struct Val {
  using type = E;
};
template <>
struct Val<uint16_t> {
  using type = int32_t;
};

// Four consecutive stored elements (16-byte aligned for 4-byte types,
// 8-byte aligned for 16-bit ones) as the value vector.
__device__ __forceinline__ float4 ld4e(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ int4 ld4e(const int32_t* p) { return *reinterpret_cast<const int4*>(p); }
__device__ __forceinline__ int4 ld4e(const uint16_t* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  return make_int4((int)(u.x & 0xffffu), (int)(u.x >> 16), (int)(u.y & 0xffffu), (int)(u.y >> 16));
}

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(long long v) { return (double)v; }

// Exact differences for TD-type sums: FP64 of two FP32 values, or int64.
__device__ __forceinline__ double dif(float a, float b) { return (double)a - (double)b; }
__device__ __forceinline__ long long dif(int32_t a, int32_t b) { return (long long)a - (long long)b; }

__device__ __forceinline__ void atomic_add_acc(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_acc(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

// v added to a 64-bit accumulator in SHARED memory with native 32-bit atomics
// (the 64-bit shared atomic add measured slower on GB300): the low word takes
// v's low half and reports whether this addition wrapped it, the high word
// then takes v's high half plus that carry.  Every thread accounts for
// exactly its own carry, so the sum is exact modulo 2^64.  p is 8-byte
// aligned (little-endian words).
__device__ __forceinline__ void atomic_add_shared64(long long* p, long long v) {
  unsigned* w = reinterpret_cast<unsigned*>(p);
  const unsigned lo = (unsigned)v;
  const unsigned hi = (unsigned)((unsigned long long)v >> 32);
  const unsigned old = atomicAdd(w, lo);
  const unsigned up = hi + ((old + lo < old) ? 1u : 0u);
  if (up) atomicAdd(w + 1, up);
}
__device__ __forceinline__ void atomic_add_shared64(double* p, double v) { atomicAdd(p, v); }

template <class A>
__device__ __forceinline__ A shfl_down_a(A v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

template <class A>
__device__ __forceinline__ Key<A> shfl_key(const Key<A>& k, int src) {
  Key<A> r;
  r.d = __shfl_sync(0xffffffffu, k.d, src);
  r.slot = __shfl_sync(0xffffffffu, k.slot, src);
  r.cand = __shfl_sync(0xffffffffu, k.cand, src);
  return r;
}

// Warp-wide lexicographic minimum; the result is valid in every lane.
template <class A>
__device__ __forceinline__ Key<A> warp_min_key(Key<A> k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Key<A> other;
    other.d = __shfl_xor_sync(0xffffffffu, k.d, o);
    other.slot = __shfl_xor_sync(0xffffffffu, k.slot, o);
    other.cand = __shfl_xor_sync(0xffffffffu, k.cand, o);
    if (key_less(other, k)) k = other;
  }
  return k;
}

template <class A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- timers
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------- mbarrier / TMA
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete.  Gives up after
// limit_ns (returns false) or as soon as *abort becomes nonzero.  The waits
// that let a CTA's own bulk copies land before it exits keep the default
// limit: those copies complete whatever the caller's limit is.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

// 1-D bulk copy global -> shared, completion signalled on *bar (tx bytes).
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Barrier among the consumer warps only (the producer warp runs its own
// loop), built on an mbarrier with one arrival per warp so that the wait is
// bounded like every other wait.  `phase` is the calling thread's copy of
// the barrier phase.  Returns false when the wait gave up.
__device__ __forceinline__ bool cons_sync(uint64_t* bar, uint32_t& phase, volatile int* abort,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
  const bool ok = mbar_wait(bar, phase, abort, limit_ns);
  phase ^= 1u;
  __syncwarp();
  return ok;
}

// Release-ordered atomic increment and acquire-ordered load at GPU scope.
__device__ __forceinline__ void atom_add_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier over co-resident CTAs on a monotonic arrival counter:
// the e-th barrier of the launch (epoch e = 0, 1, ...; every CTA counts its
// own) completes when *count reaches (e + 1) * gridDim.x, so no reset and
// no second word are needed.  Thread 0 of each CTA arrives with a release
// increment and polls with acquire loads.  Returns false (in every thread
// of the CTA) when the wait exceeded limit_ns -- then st->error =
// kErrTimeout -- or another CTA had already failed.  *count starts at 0.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& epoch, KmState* st,
                                             int* s_ok, unsigned long long limit_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (epoch + 1u) * gridDim.x;
    atom_add_release_gpu(count, 1u);
    if ((int)(ld_acquire_gpu(count) - target) < 0) {
      const unsigned long long t0 = globaltimer();
      while ((int)(ld_acquire_gpu(count) - target) < 0) {
        if (*(volatile int*)&st->error) {
          ok = 0;
          break;
        }
        if (globaltimer() - t0 > limit_ns) {
          atomicExch(&st->error, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    *s_ok = ok;
  }
  ++epoch;
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ int4 lds4(const int32_t* p) { return *reinterpret_cast<const int4*>(p); }

}  // namespace km

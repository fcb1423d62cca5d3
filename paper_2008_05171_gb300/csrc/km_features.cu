// km_features.cu -- the on-the-fly distance form of the method: BUILD
// (Alg. 1) and FastPAM1 SWAP (Alg. 3) over bf16 feature vectors with
// Euclidean distances computed in every pass instead of read from an n x n
// matrix (the paper computes distances on demand when the matrix does not
// fit, Sec. 4.8).
//
// Pass kernel k_feat_pass (one persistent CTA per SM, warp-specialised):
//   warp 0      producer: 1-D bulk copies of a 128-candidate tile (A), of
//               128-point blocks (B) into a ring of as many stages as shared
//               memory holds (freed by the MMA's completion), and of the
//               blocks' cache entries into a separate 4-stage ring (freed
//               by the epilogue), all with mbarrier completion;
//   warp 1      allocates tensor memory and issues the tcgen05 MMAs:
//               G = X_c X_o^T, BF16 inputs, FP32 accumulation, into one of
//               four 128-column TMEM accumulators;
//   warps 2-17  epilogue, four warpgroups of 32 columns each: read the
//               MMA output from TMEM and test every pair against its
//               point's threshold,
//               d(o,c)^2 < d^2(o)  <=>  g - |x_c|^2/2 > (|x_o|^2 - d^2(o))/2,
//               folded into the product itself (the operands carry
//               |x_c|^2/2 and the threshold in 16 extra columns, see
//               FeatArgs), so the sign bit of each output is the test,
//               funnel-shifted into a 16-bit lane mask (one shift a pair);
//               the pairs that pass (rare) are walked lane by lane (or, in
//               a group where some lane has many, with predication) and
//               take d = sqrt(|x_c|^2 + |x_o|^2 - 2 g) (hardware square
//               root):
//               SWAP:  Eq. (7) per-slot terms into per-candidate slot
//                      accumulators in shared memory, the shared term into
//                      a register sum;
//               BUILD: min(d - d_n, 0) summed in a register (step 0: every
//                      d).
// Every sum is exact fixed point: each distance enters as round(x 2^q), with
// q chosen per call so that the diameter of the data's bounding box is
// below 2^25 units (half the FP32 resolution of the largest distance); the
// per-slot accumulators are 32-bit words in shared memory whose wrap-arounds
// are counted in a global carry table, so every sum is an exact 64-bit
// integer, independent of the order of the atomic additions.
// The per-point cache (nearest, d_n, d_s) is computed exactly with FP32
// direct differences sum (x - y)^2 (cache, apply and BUILD commit kernels),
// so the bf16 Gram form only decides which candidate rows see a hit; its
// error near the case boundaries costs at most the error itself because the
// change function of Eq. (5) is continuous in d(o, c) at d_n and d_s.
#define KM_SRC_ID 5  // names this file in bounds-check reports
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"
#include "km_tc.cuh"

namespace km {

constexpr int kFeatEpiWarps = 16;
constexpr int kFeatThreads = (2 + kFeatEpiWarps) * 32;
constexpr int kFeatMaxK = 224;       // shared accumulators: 128 x k x 4 B
constexpr int kFeatMaxD = 256;
constexpr int kFeatMaxGrid = 160;    // pass CTAs (one per SM), carry table rows
constexpr int kFeatUnitBits = 25;    // a distance below the box diameter < 2^25 units

struct FeatArgs {
  // Operands of the pass, n_pad rows of dk = d + 16 bf16 columns each in
  // the tensor cores' core-matrix layout:
  //   A (candidate role): [-x_c, h1, h2, h3, 1, 1, 1, 0...]
  //   B (point role):     [ x_o, 1, 1, 1, t1, t2, t3, 0...]
  // with h1 + h2 + h3 = |x_c|^2 / 2 and t1 + t2 + t3 = thr[o] exactly (three
  // bf16 pieces of an FP32 value), so the product is
  //   A B^T = -x_c.x_o + |x_c|^2/2 + thr[o],
  // negative exactly when the pair passes the threshold test below.
  const uint16_t* XpA;
  uint16_t* XpB;        // its t columns follow every change of thr
  int dk;
  const uint16_t* X;    // features, row-major (ldx)
  long long ldx;
  int n, d, k, n_pad;
  const float* norms;   // |x|^2, n_pad
  // per-point cache (n_pad, padding sentinels)
  int32_t* near;
  int32_t* sec;
  float* dn;
  float* ds;
  float* dn2;
  float* ds2;
  float* thr;           // hit threshold of each point: (|x_o|^2 - d^2)/2 with
                        // d = d_s (SWAP) or d_n (BUILD); +inf on padding
  uint8_t* is_med;
  int32_t* med;
  long long* removal;   // [2][k_pad] removal loss, fixed point (units 2^-q)
  double* td2;          // [2]
  int k_pad;
  int fq;               // fixed-point exponent q: a distance x enters as round(x 2^q)
  unsigned* carry;      // [kFeatMaxGrid][kTileM][k_pad] wrap-arounds of the
                        // 32-bit per-slot accumulators (zero between tiles)
  float* range;         // [2][d] per-dimension minimum and maximum (scale)
  KmState* st;
  void* partials;       // Key<double>[kMaxGrid]
  double* gains;        // BUILD gains per step
  void* trace;
  int trace_cap;
  int mode;             // kModeSwap / kModeBuild
  int build_first;
  double tol;
  // Incremental BUILD (steps >= 1): the points whose d_n the last commit
  // lowered (every point after step 0), listed by that commit in any order:
  // their B-operand rows (XpL, the threshold columns zero during BUILD so
  // that every Gram entry is the same in every pass), |x_o|^2, a threshold
  // on the MMA output below which the pair may change the gain, and d_n
  // before and after the commit in fixed point (0 before step 0's commit);
  // bgain holds every candidate's gain sum_o min(d - d_n, 0) in fixed point.
  int incremental;
  uint16_t* XpL;
  float* lno;
  float* lthr;
  int* lqo;
  int* lqn;
  unsigned* lcnt;       // [0] entries in the list (cleared by the pass that reads
                        // it); as u64 [1] the rows every update pass streamed
  long long* bgain;
  // Incremental SWAP (k >= 2): the same list, one entry per point whose
  // cache entry a swap changed (every point for the first pass), holding
  // the new entry (lqo = d_n, lqn = d_s in fixed point) and, after a swap,
  // the old one (lqo2, lqn2; lqo2 shares lno's storage), lnear = new
  // nearest slot | old nearest slot << 16 | 1 << 31 when the old entry is
  // there, lthr = the test's bound on the MMA output from the larger d_s;
  // the list rows' threshold columns carry |x_o|^2 / 2, so the output is
  // d^2 / 2.  sg[i][c] and ss[c] are the per-slot and shared sums of
  // Eq. (7) of every candidate (magnitudes, fixed point), kept across passes.
  int swap_incremental;
  int* lnear;
  int* lqo2;
  int* lqn2;
  long long* sg;        // [k_pad][n_pad], slot-major
  long long* ss;        // [n_pad]
  // Symmetric dense pass: every candidate's distance sum (fixed point),
  // from its own tile's rows and the column sums of the tiles before it.
  unsigned long long* gsym;  // [n_pad]
};

// Pass of the incremental BUILD: the gain change of every candidate from
// the listed points (k_feat_pass with the list as the point blocks).
constexpr int kModeBuildUpd = 2;
// Pass of the incremental SWAP: the Eq. (7) sums of every candidate moved
// by the listed old and new cache entries, then every candidate's Delta.
constexpr int kModeSwapUpd = 3;
// Dense pass (first BUILD step, the k = 1 swap) with each Gram tile pair
// computed once: candidate tile t streams only the point blocks b >= t;
// every pair's distance goes to its row's sum (candidate c, point o) and,
// for b > t, to its column's sum (candidate o, point c), d being
// symmetric.  The totals meet in a global array; the last CTA takes the
// least.
constexpr int kModeBuildSym = 4;

// Adds a signed x (|x| < 2^31) to the 32-bit word w of a sum whose value is
// w + 2^32 * carry (carry a signed count in two's complement).
__device__ __forceinline__ void add_signed_word(unsigned* w, unsigned* carry,
                                                volatile unsigned char* flag, int x) {
  const unsigned u = (unsigned)x;
  const unsigned old = atomicAdd(w, u);
  const bool wrap = old + u < old;
  if (x > 0 && wrap) {
    atomicAdd(carry, 1u);
    *flag = 1;
  } else if (x < 0 && !wrap) {
    atomicAdd(carry, 0xffffffffu);
    *flag = 1;
  }
}

constexpr int kFeatAccBufs = 4;     // TMEM accumulators of kTileN columns
constexpr int kFeatMetaStages = 4;  // ring of per-block point caches
constexpr int kFeatMaxBStages = 4;  // ring of point blocks (as many as fit)

struct FeatLayout {
  size_t bars, flags, wkeys, rl, acc, red, tslot, rowc, meta, a, stages, stage_bytes, meta_bytes,
      total;
  int bst;  // point-block stages
};

__host__ __device__ inline FeatLayout feat_layout(int d, int k) {
  FeatLayout L;
  size_t o = 0;
  L.bars = o;
  o += 8 * (2 + 2 * kFeatMaxBStages + 2 * kFeatMetaStages + 2 * kFeatAccBufs + 1);
  L.flags = o;
  o += 32;
  L.tslot = o;
  o += 16;
  L.rowc = o;  // per candidate row: a carry of its slot accumulators happened
  o += kTileM;
  o = (o + 15) / 16 * 16;
  L.wkeys = o;
  o += 16 * 16;
  L.rl = o;
  o += 8 * (size_t)k;
  L.acc = o;  // SWAP: slot table; symmetric pass: column partials + counters
  const size_t sym_bytes = 8 * (size_t)kFeatMetaStages * kTileN + 4 * kFeatMetaStages;
  o += (4 * (size_t)kTileM * k > sym_bytes) ? 4 * (size_t)kTileM * k : sym_bytes;
  o = (o + 7) / 8 * 8;
  L.red = o;
  o += 8 * (size_t)kTileM * (kFeatEpiWarps / 4 - 1);
  o = (o + 127) / 128 * 128;
  L.meta = o;
  L.meta_bytes = 6 * 4 * kTileN;  // per-block point data: up to six 4-byte arrays
  o += L.meta_bytes * kFeatMetaStages;
  o = (o + 1023) / 1024 * 1024;
  L.a = o;
  o += (size_t)kTileM * d * 2;
  L.stages = o;
  L.stage_bytes = (size_t)kTileN * d * 2;
  const size_t cap = 227 * 1024;
  int bst = (o < cap) ? (int)((cap - o) / L.stage_bytes) : 0;
  if (bst > kFeatMaxBStages) bst = kFeatMaxBStages;
  if (bst < 1) bst = 1;  // then total > cap: the host rejects the shape
  L.bst = bst;
  o += L.stage_bytes * bst;
  L.total = o;
  return L;
}

__device__ __forceinline__ float bf(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }

// Three bf16 pieces whose sum is the FP32 value v exactly (each piece takes
// the next eight significant bits; a non-finite v goes whole into the
// first piece).
__device__ __forceinline__ void split3_bf16(float v, uint16_t* p) {
  if (!(v - v == 0.f)) {  // inf or NaN
    p[0] = (uint16_t)(__float_as_uint(v) >> 16);
    p[1] = p[2] = 0;
    return;
  }
  float r = v;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const __nv_bfloat16 h = __float2bfloat16_rn(r);
    p[q] = __bfloat16_as_ushort(h);
    r = r - __bfloat162float(h);  // exact: r and h agree in their leading bits
  }
}

// Offset (bf16 elements) of the 8-column chunk kc of row o in an operand
// buffer of dk columns (core-matrix layout: [o/8][kc][o%8][8]).
__device__ __forceinline__ size_t chunk_off(int o, int kc, int dk) {
  return (((size_t)(o >> 3) * (size_t)(dk >> 3) + (size_t)kc) * 8 + (size_t)(o & 7)) * 8;
}

// The B operand's extra chunk of point o: [1, 1, 1, t1, t2, t3, 0, 0].
__device__ __forceinline__ void write_thr_cols(const FeatArgs& a, int o, float thr) {
  uint16_t t[3];
  split3_bf16(thr, t);
  const uint16_t one = 0x3F80u;  // bf16 1.0
  uint4 c;
  c.x = (uint32_t)one | ((uint32_t)one << 16);
  c.y = (uint32_t)one | ((uint32_t)t[0] << 16);
  c.z = (uint32_t)t[1] | ((uint32_t)t[2] << 16);
  c.w = 0u;
  *reinterpret_cast<uint4*>(a.XpB + chunk_off(o, a.d >> 3, a.dk)) = c;
}

// v[j] for a lane-dependent j in [0, 16): a select tree over registers.
__device__ __forceinline__ float sel16(const float* v, int j) {
  const bool b0 = j & 1, b1 = j & 2, b2 = j & 4, b3 = j & 8;
  const float a0 = b0 ? v[1] : v[0], a1 = b0 ? v[3] : v[2];
  const float a2 = b0 ? v[5] : v[4], a3 = b0 ? v[7] : v[6];
  const float a4 = b0 ? v[9] : v[8], a5 = b0 ? v[11] : v[10];
  const float a6 = b0 ? v[13] : v[12], a7 = b0 ? v[15] : v[14];
  const float c0 = b1 ? a1 : a0, c1 = b1 ? a3 : a2, c2 = b1 ? a5 : a4, c3 = b1 ? a7 : a6;
  const float e0 = b2 ? c1 : c0, e1 = b2 ? c3 : c2;
  return b3 ? e1 : e0;
}

// The fixed-point value of a distance x >= 0: x 2^q rounded to the nearest
// integer (x is below the data's diameter, so the result is below 2^25;
// clamped at 2^26 against Gram rounding).  Rounding is monotone, so every
// case comparison of Eq. (7) keeps its sign in fixed point.
__device__ __forceinline__ int fxq(float x, float scale) {
  return __float2int_rn(fminf(x * scale, 67108864.f));
}

// Distance of a Gram pair in the pass: the hardware square root (relative
// error a few ulp, far below the error of the bf16 Gram entry itself), so a
// hit costs one instruction instead of the correctly rounded sequence.
__device__ __forceinline__ float pair_dist(float d2) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(d2, 0.f)));
  return r;
}

// ------------------------------------------------------------ pass kernel
template <int MODE>
__global__ void __launch_bounds__(kFeatThreads, 1) k_feat_pass(const FeatArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  KmState* st = a.st;
  if (st->done || st->error) return;
  const unsigned long long wlim = wait_limit(st);
  const int n = a.n, d = a.dk, k = a.k;  // d: the operands' K dimension
  const FeatLayout L = feat_layout(d, k);
  const int bst = L.bst;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* a_full = bars + 0;
  uint64_t* tile_done = bars + 1;                       // epilogue finished the published tile
  uint64_t* b_full = bars + 2;                          // [kFeatMaxBStages]
  uint64_t* b_empty = b_full + kFeatMaxBStages;         // [kFeatMaxBStages], MMA commit
  uint64_t* m_full = b_empty + kFeatMaxBStages;         // [kFeatMetaStages]
  uint64_t* m_empty = m_full + kFeatMetaStages;         // [kFeatMetaStages], epilogue
  uint64_t* acc_full = m_empty + kFeatMetaStages;       // [kFeatAccBufs]
  uint64_t* acc_empty = acc_full + kFeatAccBufs;        // [kFeatAccBufs]
  uint64_t* ep_bar = acc_empty + kFeatAccBufs;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.flags);
  int* last_flag = reinterpret_cast<int*>(smem + L.flags) + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.flags) + 2;
  int* tslot = reinterpret_cast<int*>(smem + L.tslot);  // tile index ping-pong [2]
  Key<double>* wkeys = reinterpret_cast<Key<double>*>(smem + L.wkeys);
  long long* rl = reinterpret_cast<long long*>(smem + L.rl);
  unsigned* acc = reinterpret_cast<unsigned*>(smem + L.acc);
  long long* red = reinterpret_cast<long long*>(smem + L.red);
  volatile unsigned char* rowc = smem + L.rowc;
  unsigned char* metas = smem + L.meta;
  unsigned char* sA = smem + L.a;
  unsigned char* stages = smem + L.stages;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rb = st->rb;
  const int ntiles = a.n_pad / kTileM;
  // the update pass streams the listed points only (read before any block
  // moves; the commit that wrote the list finished before this launch)
  constexpr bool kList = (MODE == kModeBuildUpd || MODE == kModeSwapUpd);
  constexpr bool kSwapLike = (MODE == kModeSwap || MODE == kModeSwapUpd);
  constexpr bool kSym = (MODE == kModeBuildSym);
  const int nlist =
      kList ? (int)min(__ldcg(a.lcnt), (unsigned)(MODE == kModeSwapUpd ? 2 * a.n : a.n)) : 0;
  const int nblocks = kList ? (nlist + kTileN - 1) / kTileN : a.n_pad / kTileN;
  const uint16_t* Bsrc = kList ? a.XpL : a.XpB;
  const uint32_t tile_bytes = (uint32_t)(kTileM * d * 2);

  if (kSwapLike && blockIdx.x == 0) {
    long long* rnext = a.removal + (size_t)(rb ^ 1) * a.k_pad;
    for (int i = tid; i < k; i += blockDim.x) rnext[i] = 0;
    if (tid == 0) a.td2[rb ^ 1] = 0.0;
  }
  if (!kSwapLike && blockIdx.x == 0 && tid == 0) st->build_td_d = 0.0;
  if (tid == 0) {
    mbar_init(a_full, 1);
    mbar_init(tile_done, kFeatEpiWarps);
    for (int q = 0; q < kFeatMaxBStages; ++q) {
      mbar_init(&b_full[q], 1);
      mbar_init(&b_empty[q], 1);
    }
    for (int q = 0; q < kFeatMetaStages; ++q) {
      mbar_init(&m_full[q], 1);
      mbar_init(&m_empty[q], kFeatEpiWarps);
    }
    for (int q = 0; q < kFeatAccBufs; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], kFeatEpiWarps);
    }
    mbar_init(ep_bar, kFeatEpiWarps);
    abort_flag[0] = 0;
    *last_flag = 0;
    fence_barrier_init();
  }
  if (kSwapLike) {
    const long long* rsrc = a.removal + (size_t)rb * a.k_pad;
    for (int i = tid; i < k; i += blockDim.x) rl[i] = rsrc[i];
    for (int i = tid; i < kTileM * k; i += blockDim.x) acc[i] = 0u;
  }
  for (int i = tid; i < kTileM; i += blockDim.x) rowc[i] = 0;
  // symmetric pass: per meta stage, the block's 128 column sums and the
  // count of epilogue warps that added theirs (the last one flushes)
  unsigned long long* colp = reinterpret_cast<unsigned long long*>(smem + L.acc);
  unsigned* colc = reinterpret_cast<unsigned*>(colp + kFeatMetaStages * kTileN);
  if (kSym) {
    for (int i = tid; i < kFeatMetaStages * kTileN; i += blockDim.x) colp[i] = 0ull;
    if (tid < kFeatMetaStages) colc[tid] = 0u;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kFeatAccBufs * kTileN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  Key<double> wbest;
  wbest.d = Tr<float>::g_high();
  wbest.slot = INT_MAX;
  wbest.cand = INT_MAX;

  if (warp == 0) {
    // ============================================================ producer
    if (lane == 0) {
      long long gb = 0;
      bool ok = true;
      uint32_t bused = 0, bph = 0, mused = 0, mph = 0;
      for (int seq = 0; ok; ++seq) {
        unsigned tile = atomicAdd(&st->tile_next, 1u);
        const int t = (tile < (unsigned)ntiles) ? (int)tile : -1;
        // publish a tile only after the epilogue finished the previous one:
        // no waiter on a_full can fall two phases behind, and sA is free
        if (seq > 0 && !mbar_wait(tile_done, (uint32_t)((seq - 1) & 1), abort_flag, wlim)) {
          ok = false;
          break;
        }
        tslot[seq & 1] = t;
        if (t < 0) {
          mbar_arrive(a_full);
          break;
        }
        mbar_arrive_expect_tx(a_full, tile_bytes);
        bulk_g2s(sA, a.XpA + (size_t)t * kTileM * d, tile_bytes, a_full);
        for (int b = kSym ? t : 0; b < nblocks; ++b, ++gb) {
          const int s = (int)(gb % bst);
          const uint32_t ph = (uint32_t)((gb / bst) & 1);
          if (!mbar_wait(&b_empty[s], ph ^ 1u, abort_flag, wlim)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&b_full[s], tile_bytes);
          bused |= 1u << s;
          bph = (bph & ~(1u << s)) | (ph << s);
          bulk_g2s(stages + (size_t)s * L.stage_bytes, Bsrc + (size_t)b * kTileN * d, tile_bytes,
                   &b_full[s]);
          const int ms = (int)(gb % kFeatMetaStages);
          const uint32_t mp = (uint32_t)((gb / kFeatMetaStages) & 1);
          if (!mbar_wait(&m_empty[ms], mp ^ 1u, abort_flag, wlim)) {
            ok = false;
            break;
          }
          unsigned char* meta = metas + (size_t)ms * L.meta_bytes;
          mbar_arrive_expect_tx(&m_full[ms], (uint32_t)((MODE == kModeSwapUpd ? 6 : 5) * 4 * kTileN));
          mused |= 1u << ms;
          mph = (mph & ~(1u << ms)) | (mp << ms);
          const size_t o0 = (size_t)b * kTileN;
          if (MODE == kModeBuildUpd) {
            bulk_g2s(meta, a.lno + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 512, a.lthr + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1024, a.lqo + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1536, a.lqn + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 2048, a.lqn + o0, 4 * kTileN, &m_full[ms]);  // keeps the byte count
          } else if (MODE == kModeSwapUpd) {
            bulk_g2s(meta, a.lqo2 + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 512, a.lthr + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1024, a.lqo + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1536, a.lqn + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 2048, a.lnear + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 2560, a.lqn2 + o0, 4 * kTileN, &m_full[ms]);
          } else {
            bulk_g2s(meta, a.norms + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 512, a.thr + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1024, a.dn + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 1536, a.ds + o0, 4 * kTileN, &m_full[ms]);
            bulk_g2s(meta + 2048, a.near + o0, 4 * kTileN, &m_full[ms]);
          }
        }
      }
      if (!ok) {
        abort_flag[0] = 1;
        atomicExch(&st->error, kErrTimeout);
        // wait (bounded) for this thread's own copies still in flight
        volatile int never = 0;
        for (int q = 0; q < kFeatMaxBStages; ++q)
          if (bused & (1u << q)) (void)mbar_wait(&b_full[q], (bph >> q) & 1u, &never);
        for (int q = 0; q < kFeatMetaStages; ++q)
          if (mused & (1u << q)) (void)mbar_wait(&m_full[q], (mph >> q) & 1u, &never);
      }
    }
  } else if (warp == 1) {
    // ============================================================ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc_bf16(kTileM, kTileN);
      const uint32_t lbo = 128, sbo = 16u * (uint32_t)d;
      long long gb = 0;
      long long issued = 0;  // blocks with MMAs in flight on the accumulators
      for (int seq = 0;; ++seq) {
        if (!mbar_wait(a_full, (uint32_t)(seq & 1), abort_flag, wlim)) break;
        const int t = tslot[seq & 1];
        if (t < 0) break;
        tc_fence_after();
        bool ok = true;
        for (int b = kSym ? t : 0; b < nblocks; ++b, ++gb) {
          const int s = (int)(gb % bst);
          const int buf = (int)(gb % kFeatAccBufs);
          if (!mbar_wait(&b_full[s], (uint32_t)((gb / bst) & 1), abort_flag, wlim) ||
              !mbar_wait(&acc_empty[buf], (uint32_t)(((gb / kFeatAccBufs) & 1) ^ 1), abort_flag, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(sA);
          const uint32_t sb = smem_u32(stages + (size_t)s * L.stage_bytes);
          for (int ks = 0; ks < d / 16; ++ks)
            umma_bf16(tmem + (uint32_t)(buf * kTileN), make_sdesc(sa + ks * 256, lbo, sbo),
                      make_sdesc(sb + ks * 256, lbo, sbo), idesc, ks > 0 ? 1u : 0u);
          umma_commit(&acc_full[buf]);
          umma_commit(&b_empty[s]);
          ++issued;
        }
        if (!ok) break;
      }
      if (abort_flag[0] && issued > 0) {  // let issued MMAs finish before exit
        volatile int never = 0;
        const long long lastb = gb - 1;
        (void)mbar_wait(&acc_full[lastb % kFeatAccBufs],
                        (uint32_t)((lastb / kFeatAccBufs) & 1), &never);
      }
    }
  } else {
    // ============================================================ epilogue
    const int ew = warp - 2;              // 0..15
    const int quarter = warp & 3;         // TMEM lanes 32*quarter..+31
    const int group = ew >> 2;            // columns 32*group..+31
    const int r = quarter * 32 + lane;    // candidate row within the tile
    const int col0 = group * 32;
    unsigned* arow = acc + (size_t)r * k;
    unsigned* crow = a.carry + ((size_t)blockIdx.x * kTileM + r) * a.k_pad;
    const float scale = __int_as_float((127 + a.fq) << 23);                 // 2^q
    const double unit = __longlong_as_double((long long)(1023 - a.fq) << 52);  // 2^-q
    uint32_t eph = 0;
    long long gb = 0;
    bool ok = true;
    for (int seq = 0; ok; ++seq) {
      if (!mbar_wait(a_full, (uint32_t)(seq & 1), abort_flag, wlim)) {
        ok = false;
        break;
      }
      const int t = tslot[seq & 1];
      if (t < 0) break;
      const int c = t * kTileM + r;
      const bool cvalid = (c < n) && !a.is_med[c];
      const float nc = (c < n) ? a.norms[c] : 0.f;
      // d(o,c)^2 < d^2(o)  <=>  g - |x_c|^2/2 > (|x_o|^2 - d^2(o))/2 = thr[o]
      // <=>  v = |x_c|^2/2 + thr[o] - g < 0, and v is what the MMA produced
      const float hc = 0.5f * nc;
      long long sh = 0;  // fixed point: the BUILD gain's sum or the SWAP shared term
      for (int b = kSym ? t : 0; b < nblocks; ++b, ++gb) {
        const int buf = (int)(gb % kFeatAccBufs);
        const int ms = (int)(gb % kFeatMetaStages);
        if (!mbar_wait(&acc_full[buf], (uint32_t)((gb / kFeatAccBufs) & 1), abort_flag, wlim) ||
            !mbar_wait(&m_full[ms], (uint32_t)((gb / kFeatMetaStages) & 1), abort_flag, wlim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTileN + col0), v);
        tmem_ld_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        const unsigned char* meta = metas + (size_t)ms * L.meta_bytes;
        const float* m_no = reinterpret_cast<const float*>(meta);
        const float* m_thr = reinterpret_cast<const float*>(meta + 512);
        const float* m_dn = reinterpret_cast<const float*>(meta + 1024);
        const float* m_ds = reinterpret_cast<const float*>(meta + 1536);
        const int* m_near = reinterpret_cast<const int*>(meta + 2048);
        // one pair (o = column col, candidate c = this thread's row) that
        // passed the threshold test; g = x_c.x_o recovered from v, then the
        // exact case split on d = sqrt(d^2).  Eq. (7) in fixed point: the
        // slot term (d_n - d_s, or d - d_s clamped at its case boundary
        // d = d_s where it is 0) is accumulated as its magnitude, the shared
        // term d - d_n as the magnitude d_n - d.
        auto hit = [&](int col, float v) {
          const float g = (hc + m_thr[col]) - v;
          const float d2 = fmaf(-2.f, g, nc + m_no[col]);
          const float dd = pair_dist(d2);
          const float dn_ = m_dn[col];
          const int ddq = fxq(dd, scale), dnq = fxq(dn_, scale);
          if (MODE == kModeSwap) {
            const int dsq = fxq(m_ds[col], scale);
            const int sl = m_near[col];
            const bool inner = dd < dn_;
            const int mag = inner ? dsq - dnq : max(dsq - ddq, 0);
            if (mag > 0 && KM_INB(a.st, sl, a.k)) {
              const unsigned old = atomicAdd(arow + sl, (unsigned)mag);
              if (old + (unsigned)mag < old) {  // this addition wrapped the word
                atomicAdd(crow + sl, 1u);
                rowc[r] = 1;
              }
            }
            if (inner) sh += dnq - ddq;
          } else if (dd < dn_) {
            sh += dnq - ddq;
          }
        };
        // incremental SWAP: listed point at column col, d^2 = 2 v (its
        // threshold columns carry |x_o|^2 / 2); Eq. (7)'s terms of its new
        // cache entry added and, after a swap, those of its old entry
        // subtracted, each classified in fixed point from the same d
        auto hit_upd = [&](int col, float vv) {
          const int* mq = reinterpret_cast<const int*>(meta);
          const int ddq = fxq(pair_dist(2.f * vv), scale);
          const unsigned pk = (unsigned)m_near[col];
          const int dnq = mq[256 + col], dsq = mq[384 + col];
          const int sl = (int)(pk & 0xffffu);
          long long dsh = 0;
          int mag = 0;
          if (ddq < dnq) {
            dsh = dnq - ddq;
            mag = dsq - dnq;
          } else if (ddq < dsq) {
            mag = dsq - ddq;
          }
          if (pk >> 31) {
            const int sl2 = (int)((pk >> 16) & 0x7fffu);
            const int dnq2 = mq[col], dsq2 = mq[640 + col];
            int mag2 = 0;
            if (ddq < dnq2) {
              dsh -= dnq2 - ddq;
              mag2 = dsq2 - dnq2;
            } else if (ddq < dsq2) {
              mag2 = dsq2 - ddq;
            }
            if (sl2 == sl) {
              mag -= mag2;
            } else if (mag2 > 0 && KM_INB(a.st, sl2, a.k)) {
              add_signed_word(arow + sl2, crow + sl2, rowc + r, -mag2);
            }
          }
          sh += dsh;
          if (mag != 0 && KM_INB(a.st, sl, a.k)) add_signed_word(arow + sl, crow + sl, rowc + r, mag);
        };
        // incremental BUILD: listed point o (column col), v = |x_c|^2/2 -
        // x_c.x_o (zero threshold columns), so d^2 = |x_o|^2 + 2 v; the pair
        // can change the gain only when d is below the larger of its old and
        // new d_n (lthr is that bound with a margin, so the test lets through
        // a superset); the change min(d - dn_new, 0) - min(d - dn_old, 0) is
        // exact in fixed point, and zero for the pairs the margin adds
        auto hit_b = [&](int col, float vv) {
          const int* mq = reinterpret_cast<const int*>(meta);
          const int ddq = fxq(pair_dist(fmaf(2.f, vv, m_no[col])), scale);
          sh += (long long)(min(ddq - mq[384 + col], 0) - min(ddq - mq[256 + col], 0));
        };
        if (kSym) {
          // every pair once: x[j] = d(c, o_j) in fixed point (0 where the
          // row or the column is padding) into this row's sum
          const int colg = b * kTileN + col0;
          unsigned x[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float g = (hc + m_thr[col0 + j]) - v[j];
            const float d2 = fmaf(-2.f, g, nc + m_no[col0 + j]);
            x[j] = (c < n && colg + j < n) ? (unsigned)fxq(pair_dist(d2), scale) : 0u;
            sh += x[j];
          }
          if (b != t) {
            // column sums over the warp's 32 rows (each below 2^31: 32
            // terms below 2^26): at every halving step a lane keeps the
            // half of its columns selected by its lane bit and adds the
            // partner's copy of that half, so lane j ends with column j
#pragma unroll
            for (int h = 16; h >= 1; h >>= 1) {
              const bool up = (lane & h) != 0;
#pragma unroll
              for (int i = 0; i < h; ++i) {
                const unsigned keep = up ? x[i + h] : x[i];
                const unsigned send = up ? x[i] : x[i + h];
                x[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
              }
            }
            unsigned long long* cp = colp + (size_t)ms * kTileN;
            atomicAdd(cp + col0 + lane, (unsigned long long)x[0]);
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) {
              __threadfence_block();
              last = (atomicAdd(colc + ms, 1u) == (unsigned)kFeatEpiWarps - 1u) ? 1u : 0u;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
              // every warp's sums of this block are in: add the block's
              // columns to those points' totals as candidates, clear the
              // stage's partials (reused after the stage is released)
              __threadfence_block();
#pragma unroll
              for (int q = 0; q < kTileN / 32; ++q) {
                const int col = q * 32 + lane;
                const unsigned long long vsum = atomicExch(cp + col, 0ull);
                if (vsum) atomicAdd(a.gsym + (size_t)b * kTileN + col, vsum);
              }
              if (lane == 0) atomicExch(colc + ms, 0u);
            }
          }
        } else if (MODE == kModeBuild && a.build_first) {
          // every pair (thr = 0 before the first BUILD step)
          const int colg = b * kTileN + col0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float g = (hc + m_thr[col0 + j]) - v[j];
            const float d2 = fmaf(-2.f, g, nc + m_no[col0 + j]);
            sh += (colg + j < n) ? fxq(pair_dist(d2), scale) : 0;
          }
        } else {
#pragma unroll
          for (int g16 = 0; g16 < 2; ++g16) {
            // fast path: bit j of the lane mask is the sign of v for column
            // j (set: a hit), shifted in from column 15 down to 0 with one
            // funnel shift per pair; rows that are not candidates see none
            unsigned mask = 0;
            if (MODE == kModeSwapUpd || MODE == kModeBuildUpd) {
              // explicit test against each entry's bound: the sign of
              // v - bound (negative exactly when v < bound), funnel-shifted
              // as in the plain pass; entries past the list's end see none,
              // and in SWAP rows c >= n (every row c < n counts: a medoid
              // swapped out later is a candidate again)
              const int cbase = b * kTileN + col0 + g16 * 16;
#pragma unroll
              for (int j = 15; j >= 0; --j)
                mask = __funnelshift_l(
                    __float_as_uint(v[g16 * 16 + j] - m_thr[col0 + g16 * 16 + j]), mask, 1);
              const int left = nlist - cbase;
              if (left < 16) mask &= (left > 0) ? ((1u << left) - 1u) : 0u;
              // BUILD: only candidates (a medoid's gain is never used again)
              if (MODE == kModeSwapUpd ? c >= n : !cvalid) mask = 0;
            } else {
#pragma unroll
              for (int j = 15; j >= 0; --j)
                mask = __funnelshift_l(__float_as_uint(v[g16 * 16 + j]), mask, 1);
              if (!cvalid) mask = 0;
            }
            const unsigned most = __reduce_max_sync(0xffffffffu, (unsigned)__popc(mask));
            if (most == 0) continue;
            const int cb = col0 + g16 * 16;
            if (most > 4) {
              // dense group: every column, predicated on its bit
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if ((mask >> j) & 1u) {
                  if (MODE == kModeSwapUpd)
                    hit_upd(cb + j, v[g16 * 16 + j]);
                  else if (MODE == kModeBuildUpd)
                    hit_b(cb + j, v[g16 * 16 + j]);
                  else
                    hit(cb + j, v[g16 * 16 + j]);
                }
            } else {
              // sparse group: each lane walks its own hits
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                if (MODE == kModeSwapUpd)
                  hit_upd(cb + j, sel16(v + g16 * 16, j));
                else if (MODE == kModeBuildUpd)
                  hit_b(cb + j, sel16(v + g16 * 16, j));
                else
                  hit(cb + j, sel16(v + g16 * 16, j));
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&m_empty[ms]);
      }
      if (!ok) break;
      // ------------------------------------------------------ tile finished
      if (group > 0) red[(group - 1) * kTileM + r] = sh;
      if (!cons_sync(ep_bar, eph, abort_flag, wlim)) {
        ok = false;
        break;
      }
      if (group == 0) {
        long long shared_part = sh;
        for (int g = 0; g < kFeatEpiWarps / 4 - 1; ++g) shared_part += red[g * kTileM + r];
        if (MODE == kModeSwap) {
          // Delta_i = removal loss of slot i - the slot's accumulated
          // magnitudes (32-bit word + 2^32 x its wrap count); Delta(c) =
          // min_i Delta_i + Delta^{+c}, all exact integers
          const bool carried = rowc[r] != 0;
          if (cvalid) {
            long long best = LLONG_MAX;
            int bi = 0;
            for (int i = 0; i < k; ++i) {
              long long t = (long long)arow[i];
              if (carried) t += (long long)__ldcg(crow + i) << 32;
              const long long vi = rl[i] - t;
              if (vi < best) {
                best = vi;
                bi = i;
              }
            }
            Key<double> ck;
            ck.d = (double)(best - shared_part) * unit;
            ck.slot = bi;
            ck.cand = c;
            if (key_less(ck, wbest)) wbest = ck;
          }
          for (int i = 0; i < k; ++i) arow[i] = 0u;
          if (carried) {
            for (int i = 0; i < k; ++i) __stcg(crow + i, 0u);
            rowc[r] = 0;
          }
        } else if (MODE == kModeSwapUpd) {
          // the kept sums of row c moved by this pass (word + 2^32 x its
          // signed carry count), then Delta(c) as in the plain pass
          const bool carried = rowc[r] != 0;
          if (c < n) {
            long long best = LLONG_MAX;
            int bi = 0;
            // the kept sums are slot-major, so the 32 rows of a warp read
            // consecutive words; eight slots' loads in flight at a time
            constexpr int U = 8;
            for (int i0 = 0; i0 < k; i0 += U) {
              long long gv[U];
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (i0 + u < k) gv[u] = __ldcg(a.sg + (size_t)(i0 + u) * a.n_pad + c);
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int i = i0 + u;
                if (i < k) {
                  long long t = (long long)arow[i];
                  if (carried) t += (long long)(int)__ldcg(crow + i) * 4294967296ll;
                  const long long gi = gv[u] + t;
                  a.sg[(size_t)i * a.n_pad + c] = gi;
                  const long long vi = rl[i] - gi;
                  if (vi < best) {
                    best = vi;
                    bi = i;
                  }
                }
              }
            }
            const long long sc = a.ss[c] + shared_part;
            a.ss[c] = sc;
            if (cvalid) {
              Key<double> ck;
              ck.d = (double)(best - sc) * unit;
              ck.slot = bi;
              ck.cand = c;
              if (key_less(ck, wbest)) wbest = ck;
            }
          }
          for (int i = 0; i < k; ++i) arow[i] = 0u;
          if (carried) {
            for (int i = 0; i < k; ++i) __stcg(crow + i, 0u);
            rowc[r] = 0;
          }
        } else if (MODE == kModeBuildUpd) {
          if (c < n) {
            const long long g = a.bgain[c] + shared_part;  // one CTA owns the tile
            a.bgain[c] = g;
            if (cvalid) {
              Key<double> ck;
              ck.d = (double)g * unit;
              ck.slot = 0;
              ck.cand = c;
              if (key_less(ck, wbest)) wbest = ck;
            }
          }
        } else if (kSym) {
          if (c < n) atomicAdd(a.gsym + c, (unsigned long long)shared_part);
        } else {
          if (cvalid) {
            Key<double> ck;
            ck.d = (double)(a.build_first ? shared_part : -shared_part) * unit;
            ck.slot = 0;
            ck.cand = c;
            if (key_less(ck, wbest)) wbest = ck;
          }
        }
      }
      if (!cons_sync(ep_bar, eph, abort_flag, wlim)) {
        ok = false;
        break;
      }
      if (lane == 0) mbar_arrive(tile_done);
    }
    if (!ok) {
      abort_flag[0] = 1;
      atomicExch(&st->error, kErrTimeout);
    }
    if (kSym) __threadfence();  // this thread's totals before the CTA's ticket
    wbest = warp_min_key(wbest);
    if (lane == 0) wkeys[ew] = wbest;
  }

  // ------------------------------------------------------------ CTA result
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kFeatAccBufs * kTileN);
  if (tid == 0) {
    Key<double> b = wkeys[0];
    for (int w = 1; w < kFeatEpiWarps; ++w)
      if (key_less(wkeys[w], b)) b = wkeys[w];
    reinterpret_cast<Key<double>*>(a.partials)[blockIdx.x] = b;
    __threadfence();
    const unsigned tk = atomicAdd(&st->ticket, 1u);
    *last_flag = (tk == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!*last_flag) return;
  __threadfence();
  if (kSym) {
    // every CTA's totals are in: the least over the non-medoid candidates,
    // eight of each thread's loads in flight
    const double unit = __longlong_as_double((long long)(1023 - a.fq) << 52);
    Key<double> b;
    b.d = Tr<float>::g_high();
    b.slot = INT_MAX;
    b.cand = INT_MAX;
    constexpr int U = 8;
    for (int c0 = tid; c0 < n; c0 += U * kFeatThreads) {
      unsigned long long tv[U];
      unsigned char mv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + u * kFeatThreads;
        tv[u] = (c < n) ? __ldcg(a.gsym + c) : 0ull;
        mv[u] = (c < n) ? a.is_med[c] : (unsigned char)1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (!mv[u]) {
          Key<double> ck;
          ck.d = (double)(long long)tv[u] * unit;
          ck.slot = 0;
          ck.cand = c0 + u * kFeatThreads;
          if (key_less(ck, b)) b = ck;
        }
    }
    b = warp_min_key(b);
    Key<double>* kk = reinterpret_cast<Key<double>*>(red);  // free after the tiles
    if (lane == 0) kk[warp] = b;
    __syncthreads();
    if (tid == 0) {
      Key<double> bb = kk[0];
      for (int w = 1; w < kFeatThreads / 32; ++w)
        if (key_less(kk[w], bb)) bb = kk[w];
      st->build_gain_d = bb.d;
      st->build_cand = bb.cand;
      st->tile_next = 0;
      st->ticket = 0;
    }
    return;
  }
  if (warp == 0) {
    Key<double> b;
    b.d = Tr<float>::g_high();
    b.slot = INT_MAX;
    b.cand = INT_MAX;
    for (int g = lane; g < (int)gridDim.x; g += 32) {
      const Key<double> v = ld_cg_key(reinterpret_cast<const Key<double>*>(a.partials) + g);
      if (key_less(v, b)) b = v;
    }
    b = warp_min_key(b);
    if (lane == 0) {
      if (!kSwapLike) {
        st->build_gain_d = b.d;
        st->build_cand = b.cand;
        if (MODE == kModeBuildUpd) {
          // rows streamed by the update passes, then an empty list for the
          // next commit
          reinterpret_cast<unsigned long long*>(a.lcnt)[1] += (unsigned long long)nlist;
          *a.lcnt = 0u;
        }
      } else {
        if (MODE == kModeSwapUpd) *a.lcnt = 0u;  // the next swap writes a new list
        st->best_d = b.d;
        st->best_i = 0;
        st->best_slot = (b.cand == INT_MAX) ? -1 : b.slot;
        st->best_cand = (b.cand == INT_MAX) ? -1 : b.cand;
        st->iter += 1;
        if (b.cand != INT_MAX && b.d < -a.tol) {
          st->accept = 1;
        } else {
          st->accept = 0;
          st->done = 1;
        }
      }
      st->tile_next = 0;
      st->ticket = 0;
    }
  }
}

// ------------------------------------------------- exact distance kernels
// Squared Euclidean distance in FP32 by direct differences.
__device__ __forceinline__ float dist2_rows(const uint16_t* x, const uint16_t* y, int d) {
  float s = 0.f;
  for (int t = 0; t < d; t += 8) {
    const uint4 a = *reinterpret_cast<const uint4*>(x + t);
    const uint4 b = *reinterpret_cast<const uint4*>(y + t);
    const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float d0 = __uint_as_float(av[q] << 16) - __uint_as_float(bv[q] << 16);
      const float d1 = __uint_as_float(av[q] & 0xffff0000u) - __uint_as_float(bv[q] & 0xffff0000u);
      s = fmaf(d0, d0, s);
      s = fmaf(d1, d1, s);
    }
  }
  return s;
}

template <class V>
__device__ __forceinline__ V fblock_sum(V v, V* scratch) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
  __syncthreads();
  V r = V(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += scratch[i];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void top2f(float v, int j, int& n1, float& d1, int& n2, float& d2) {
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

// One entry of the incremental SWAP's list at position p: point o's new
// cache entry (d_n, d_s, nearest slot) and, when has_old, the entry it had
// before the swap; the bound of the pass's test from the larger d_s (the
// MMA output v = d^2 / 2 is below it iff d is below that d_s, with a 2^-10
// relative margin on d^2); o's B-operand row with |x_o|^2 / 2 in its
// threshold columns.
__device__ __forceinline__ void swap_list_put(const FeatArgs& a, unsigned p, int o, float dn,
                                              float ds, int near, bool has_old, float dn_old,
                                              float ds_old, int near_old) {
  const float scale = __int_as_float((127 + a.fq) << 23);
  const float dsm = has_old ? fmaxf(ds, ds_old) : ds;
  a.lthr[p] = 0.5f * (dsm * dsm * (1.f + 0x1p-10f) + 0x1p-100f);
  a.lqo[p] = fxq(dn, scale);
  a.lqn[p] = fxq(ds, scale);
  a.lqo2[p] = has_old ? fxq(dn_old, scale) : 0;
  a.lqn2[p] = has_old ? fxq(ds_old, scale) : 0;
  a.lnear[p] = (int)(((unsigned)near & 0xffffu) |
                     (has_old ? ((((unsigned)near_old & 0x7fffu) << 16) | 0x80000000u) : 0u));
  const int kcs = a.dk >> 3;
  for (int kc = 0; kc < kcs; ++kc)
    *reinterpret_cast<uint4*>(a.XpL + chunk_off((int)p, kc, a.dk)) =
        *reinterpret_cast<const uint4*>(a.XpB + chunk_off(o, kc, a.dk));
  uint16_t t[3];
  split3_bf16(0.5f * a.norms[o], t);
  const uint16_t one = 0x3F80u;  // bf16 1.0
  uint4 c;
  c.x = (uint32_t)one | ((uint32_t)one << 16);
  c.y = (uint32_t)one | ((uint32_t)t[0] << 16);
  c.z = (uint32_t)t[1] | ((uint32_t)t[2] << 16);
  c.w = 0u;
  *reinterpret_cast<uint4*>(a.XpL + chunk_off((int)p, a.d >> 3, a.dk)) = c;
}

// Warp-aggregated reservation of cnt list positions per lane (cnt 0..2).
__device__ __forceinline__ unsigned list_reserve(unsigned* lcnt, unsigned cnt) {
  const int lane = threadIdx.x & 31;
  unsigned incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned base = 0;
  if (lane == 31 && total) base = atomicAdd(lcnt, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - cnt;
}

// Exact cache of every point for the current medoids (distances compared
// squared; d_n, d_s stored as FP32 square roots), removal loss and TD.
__global__ void __launch_bounds__(256) k_feat_cache(const FeatArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(sm);
  __shared__ double scratch[8];
  __shared__ int is_last;
  KmState* st = a.st;
  const int k = a.k, n = a.n, d = a.d;
  const int rb = st->rb;
  const float scale = __int_as_float((127 + a.fq) << 23);
  for (int i = threadIdx.x; i < k; i += blockDim.x) sacc[i] = 0ull;
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  double tdl = 0.0;
  if (o < n) {
    const uint16_t* xo = a.X + (size_t)o * a.ldx;
    int n1 = -1, n2 = -1;
    float q1 = 0.f, q2 = 0.f;
    for (int j = 0; j < k; ++j)
      if (KM_INB(st, a.med[j], n))
        top2f(dist2_rows(xo, a.X + (size_t)a.med[j] * a.ldx, d), j, n1, q1, n2, q2);
    const float e1 = sqrtf(q1);
    const float e2 = (n2 < 0) ? Tr<float>::high() : sqrtf(q2);
    a.near[o] = n1;
    a.sec[o] = n2;
    a.dn[o] = e1;
    a.ds[o] = e2;
    a.dn2[o] = q1;
    a.ds2[o] = (n2 < 0) ? Tr<float>::high() : q2;
    // k = 1 has no second medoid; its SWAP is a dense pass (every pair), for
    // which any finite threshold lets the Gram entries be recovered.  The
    // incremental SWAP keeps the threshold columns zero (each pair's Gram
    // entry the same in every pass) and tests explicitly.
    a.thr[o] = (n2 < 0 || a.swap_incremental) ? 0.f : 0.5f * (a.norms[o] - q2);
    write_thr_cols(a, o, a.thr[o]);
    if (n2 >= 0 && n1 >= 0)
      atomicAdd(&sacc[n1], (unsigned long long)(fxq(e2, scale) - fxq(e1, scale)));
    tdl = e1;
  } else if (o < a.n_pad) {
    a.near[o] = 0;
    a.sec[o] = 0;
    a.dn[o] = 0.f;
    a.ds[o] = 0.f;
    a.dn2[o] = Tr<float>::low();
    a.ds2[o] = Tr<float>::low();
    a.thr[o] = Tr<float>::high();
    write_thr_cols(a, o, Tr<float>::high());
  }
  if (a.swap_incremental) {  // uniform: every point's entry opens the list
    const bool put = o < n;
    const unsigned p = list_reserve(a.lcnt, put ? 1u : 0u);
    if (put && KM_INB(st, p, 2 * (long long)a.n_pad))
      swap_list_put(a, p, o, a.dn[o], a.ds[o], a.near[o], false, 0.f, 0.f, 0);
  }
  const double bs = fblock_sum(tdl, scratch);
  if (threadIdx.x == 0) atomicAdd(&a.td2[rb], bs);
  unsigned long long* rem = reinterpret_cast<unsigned long long*>(a.removal + (size_t)rb * a.k_pad);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (sacc[i] != 0ull) atomicAdd(&rem[i], sacc[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    st->td_book_d = static_cast<volatile double*>(a.td2)[rb];
    st->ticket = 0;
  }
}

// Apply the pending swap (slot i* <- candidate c*) with an incremental,
// exact cache update; removal loss and TD of the next pass on the way.
__global__ void __launch_bounds__(256) k_feat_apply(const FeatArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(sm);
  __shared__ double scratch[8];
  __shared__ int is_last;
  KmState* st = a.st;
  if (st->error || !st->accept) return;
  const int k = a.k, n = a.n, d = a.d;
  const int i_s = st->best_slot, c_s = st->best_cand;
  if (!KM_INB(st, i_s, k) || !KM_INB(st, c_s, n)) return;  // uniform for the launch
  const int rb = st->rb;
  const float scale = __int_as_float((127 + a.fq) << 23);
  for (int i = threadIdx.x; i < k; i += blockDim.x) sacc[i] = 0ull;
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  double tdl = 0.0;
  bool changed = false;
  int n1_old = 0;
  float dn_old = 0.f, ds_old = 0.f;
  if (o < n) {
    const uint16_t* xo = a.X + (size_t)o * a.ldx;
    int n1 = a.near[o], n2 = a.sec[o];
    float q1 = a.dn2[o], q2 = a.ds2[o];
    const float q1_old = q1, q2_old = q2;
    n1_old = n1;
    dn_old = a.dn[o];
    ds_old = a.ds[o];
    if (n1 == i_s || n2 == i_s) {
      n1 = -1;
      n2 = -1;
      for (int j = 0; j < k; ++j) {
        const int m = (j == i_s) ? c_s : a.med[j];
        if (!KM_INB(st, m, n)) continue;
        top2f(dist2_rows(xo, a.X + (size_t)m * a.ldx, d), j, n1, q1, n2, q2);
      }
    } else {
      const float qc = dist2_rows(xo, a.X + (size_t)c_s * a.ldx, d);
      if (qc < q1 || (qc == q1 && i_s < n1)) {
        n2 = n1;
        q2 = q1;
        n1 = i_s;
        q1 = qc;
      } else if (qc < q2 || (qc == q2 && i_s < n2)) {
        n2 = i_s;
        q2 = qc;
      }
    }
    const float e1 = sqrtf(q1), e2 = sqrtf(q2);
    changed = n1 != n1_old || q1 != q1_old || q2 != q2_old;
    a.near[o] = n1;
    a.sec[o] = n2;
    a.dn[o] = e1;
    a.ds[o] = e2;
    a.dn2[o] = q1;
    a.ds2[o] = q2;
    if (!a.swap_incremental) {
      a.thr[o] = 0.5f * (a.norms[o] - q2);
      write_thr_cols(a, o, a.thr[o]);
    }
    if (KM_INB(st, n1, k))
      atomicAdd(&sacc[n1], (unsigned long long)(fxq(e2, scale) - fxq(e1, scale)));
    tdl = e1;
  }
  if (a.swap_incremental) {  // uniform: a changed point's new entry in, old one out
    const unsigned p = list_reserve(a.lcnt, changed ? 1u : 0u);
    if (changed && KM_INB(st, p, 2 * (long long)a.n_pad))
      swap_list_put(a, p, o, a.dn[o], a.ds[o], a.near[o], true, dn_old, ds_old, n1_old);
  }
  const double bs = fblock_sum(tdl, scratch);
  if (threadIdx.x == 0) atomicAdd(&a.td2[rb ^ 1], bs);
  unsigned long long* rem =
      reinterpret_cast<unsigned long long*>(a.removal + (size_t)(rb ^ 1) * a.k_pad);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (sacc[i] != 0ull) atomicAdd(&rem[i], sacc[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    const int old = a.med[i_s];
    a.med[i_s] = c_s;
    a.is_med[old] = 0;
    a.is_med[c_s] = 1;
    const int nt = st->ntrace;
    if (nt < a.trace_cap) {
      TraceRec* tr = static_cast<TraceRec*>(a.trace) + nt;
      tr->d = st->best_d;
      tr->di = 0;
      tr->slot = i_s;
      tr->cand = c_s;
      tr->t_ns = (long long)globaltimer();
    }
    st->ntrace = nt + 1;
    st->swaps += 1;
    st->td_book_d += st->best_d;
    st->accept = 0;
    st->rb = rb ^ 1;
    st->ticket = 0;
  }
}

// BUILD commit: add the chosen point and lower d_n (exact FP32 distances).
// Incremental BUILD: every point whose d_n this commit lowered (every point
// at step 0) is appended to the list for the next update pass, its B row
// copied into XpL; the plain pass instead gets the new threshold columns.
__global__ void __launch_bounds__(256) k_feat_build_commit(const FeatArgs a) {
  __shared__ double scratch[8];
  KmState* st = a.st;
  if (st->error) return;
  const int n = a.n, d = a.d;
  const int c = st->build_cand;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const float scale = __int_as_float((127 + a.fq) << 23);  // 2^q
  double local = 0.0;
  if (c >= 0 && c < n) {
    bool listed = false;
    float old_dn = 0.f, new_dn = 0.f;
    if (o < n) {
      const float q = dist2_rows(a.X + (size_t)o * a.ldx, a.X + (size_t)c * a.ldx, d);
      float cur = q;
      if (!a.build_first && !(q < a.dn2[o])) cur = a.dn2[o];
      listed = a.build_first || q < a.dn2[o];
      old_dn = a.build_first ? 0.f : a.dn[o];
      a.dn2[o] = cur;
      a.dn[o] = sqrtf(cur);
      new_dn = a.dn[o];
      if (!a.incremental) {
        a.thr[o] = 0.5f * (a.norms[o] - cur);
        write_thr_cols(a, o, a.thr[o]);
      }
      local = sqrtf(cur);
    } else if (o < a.n_pad) {
      a.dn2[o] = Tr<float>::low();
      a.dn[o] = 0.f;
      if (!a.incremental) {
        a.thr[o] = Tr<float>::high();
        write_thr_cols(a, o, Tr<float>::high());
      }
    }
    if (a.incremental) {
      // warp-aggregated append
      const unsigned m = __ballot_sync(0xffffffffu, listed);
      if (m) {
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(a.lcnt, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (listed) {
          unsigned lt;
          asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
          const unsigned p = base + (unsigned)__popc(m & lt);
          if (KM_INB(st, p, a.n_pad)) {
            const float no = a.norms[o];
            const float dmax = fmaxf(old_dn, new_dn);
            a.lno[p] = no;
            // v = (d^2 - |x_o|^2) / 2 below this bound: d below dmax with a
            // relative margin of 2^-10 on d^2 that covers every rounding
            a.lthr[p] = 0.5f * (dmax * dmax * (1.f + 0x1p-10f) + 0x1p-100f - no);
            a.lqo[p] = a.build_first ? 0 : fxq(old_dn, scale);
            a.lqn[p] = fxq(new_dn, scale);
            const int kcs = a.dk >> 3;
            for (int kc = 0; kc < kcs; ++kc)
              *reinterpret_cast<uint4*>(a.XpL + chunk_off((int)p, kc, a.dk)) =
                  *reinterpret_cast<const uint4*>(a.XpB + chunk_off(o, kc, a.dk));
          }
        }
      }
    }
  }
  const double bs = fblock_sum(local, scratch);
  if (threadIdx.x == 0) atomicAdd(&st->build_td_d, bs);
  if (blockIdx.x == 0 && threadIdx.x == 0 && c >= 0 && c < n &&
      KM_INB(st, st->build_step, a.k)) {
    const int step = st->build_step;
    a.med[step] = c;
    a.is_med[c] = 1;
    if (a.gains) a.gains[step] = st->build_gain_d;
    st->td_book_d = a.build_first ? st->build_gain_d : st->td_book_d + st->build_gain_d;
    st->build_step = step + 1;
  }
}

// Both operand buffers of the pass from the features (see FeatArgs); thr
// starts at 0 for points (finite, so the first BUILD step can recover every
// Gram entry) and +inf on padding rows.
__global__ void k_feat_prearrange(const FeatArgs a) {
  const int dc = a.d >> 3, kcs = a.dk >> 3;
  const long long chunks = (long long)a.n_pad * kcs;
  uint16_t* XpA = const_cast<uint16_t*>(a.XpA);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < chunks;
       q += (long long)gridDim.x * blockDim.x) {
    const long long g = q / ((long long)kcs * 8);
    const long long rem = q - g * kcs * 8;
    const int kc = (int)(rem / 8), rr = (int)(rem % 8);
    const int row = (int)(g * 8 + rr);
    uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
    if (kc < dc) {
      if (row < a.n) {
        vb = *reinterpret_cast<const uint4*>(a.X + (size_t)row * a.ldx + kc * 8);
        va = make_uint4(vb.x ^ 0x80008000u, vb.y ^ 0x80008000u, vb.z ^ 0x80008000u,
                        vb.w ^ 0x80008000u);
      }
    } else if (kc == dc) {
      const float thr0 = (row < a.n) ? 0.f : Tr<float>::high();
      a.thr[row] = thr0;
      uint16_t t[3];
      split3_bf16(thr0, t);
      const uint16_t one = 0x3F80u;
      vb = make_uint4((uint32_t)one | ((uint32_t)one << 16), (uint32_t)one | ((uint32_t)t[0] << 16),
                      (uint32_t)t[1] | ((uint32_t)t[2] << 16), 0u);
      if (row < a.n) {
        uint16_t h[3];
        split3_bf16(0.5f * a.norms[row], h);
        va = make_uint4((uint32_t)h[0] | ((uint32_t)h[1] << 16),
                        (uint32_t)h[2] | ((uint32_t)one << 16),
                        (uint32_t)one | ((uint32_t)one << 16), 0u);
      }
    }
    reinterpret_cast<uint4*>(XpA)[q] = va;
    reinterpret_cast<uint4*>(a.XpB)[q] = vb;
  }
}

// Per-dimension minimum and maximum of the features (thread t of a block
// takes dimension t of every gridDim-th point), as order-preserving integer
// encodings of the float values so that integer atomics combine them.
__device__ __forceinline__ int ord_of(float v) {
  const int b = __float_as_int(v);
  return b >= 0 ? b : b ^ 0x7fffffff;
}

__global__ void k_feat_range(const FeatArgs a) {
  const int t = threadIdx.x;
  if (t >= a.d) return;
  int lo = INT_MAX, hi = INT_MIN;
  for (int o = blockIdx.x; o < a.n; o += gridDim.x) {
    const int v = ord_of(bf(a.X[(size_t)o * a.ldx + t]));
    lo = min(lo, v);
    hi = max(hi, v);
  }
  int* r = reinterpret_cast<int*>(a.range);
  atomicMin(r + t, lo);
  atomicMax(r + a.d + t, hi);
}

__global__ void k_feat_mark(const FeatArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.k) a.is_med[a.med[j]] = 1;
}

}  // namespace km

// ============================================================== host side
using namespace km;

namespace {

struct FeatWs {
  size_t st, med, is_med, near, sec, dn, ds, dn2, ds2, thr, norms, removal, td2, partials, trace,
      gains, xpa, xpb, carry, range, xpl, lno, lthr, lqo, lqn, lnear, lqn2, lcnt, bgain, sg, ss, gsym,
      total;
  int n_pad, k_pad, cap;
};

bool feat_ws(int64_t n, int d, int k, const km_options* o, FeatWs* L) {
  if (n <= 0 || k <= 0 || k > n || d <= 0 || d + 16 > kFeatMaxD || d % 16 || n > (1 << 28))
    return false;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const int n_pad = (int)((n + kTileM - 1) / kTileM * kTileM);
  const int k_pad = (k + 31) / 32 * 32;
  const int cap = (o && o->trace_capacity > 0) ? o->trace_capacity : 0;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t r = off;
    off += al(b);
    return r;
  };
  L->st = take(512);
  L->med = take(4 * (size_t)k_pad);
  L->is_med = take((size_t)n_pad);
  L->near = take(4 * (size_t)n_pad);
  L->sec = take(4 * (size_t)n_pad);
  L->dn = take(4 * (size_t)n_pad);
  L->ds = take(4 * (size_t)n_pad);
  L->dn2 = take(4 * (size_t)n_pad);
  L->ds2 = take(4 * (size_t)n_pad);
  L->thr = take(4 * (size_t)n_pad);
  L->norms = take(4 * (size_t)n_pad);
  L->removal = take(16 * (size_t)k_pad);
  L->td2 = take(16);
  L->partials = take(16 * (size_t)kMaxGrid);
  L->trace = take(sizeof(TraceRec) * (size_t)(cap > 0 ? cap : 1));
  L->gains = take(8 * (size_t)k);
  L->xpa = take((size_t)n_pad * (d + 16) * 2);
  L->xpb = take((size_t)n_pad * (d + 16) * 2);
  L->carry = take(4 * (size_t)kFeatMaxGrid * kTileM * k_pad);
  L->range = take(8 * (size_t)d);
  // incremental BUILD and SWAP: the list (BUILD: one entry per changed
  // point; SWAP: an old and a new entry each), every candidate's BUILD gain,
  // and the SWAP's per-slot and shared sums of every candidate
  L->xpl = take(2 * (size_t)n_pad * (d + 16) * 2);
  L->lno = take(8 * (size_t)n_pad);
  L->lthr = take(8 * (size_t)n_pad);
  L->lqo = take(8 * (size_t)n_pad);
  L->lqn = take(8 * (size_t)n_pad);
  L->lnear = take(8 * (size_t)n_pad);
  L->lqn2 = take(8 * (size_t)n_pad);
  L->lcnt = take(16);
  L->bgain = take(8 * (size_t)n_pad);
  const bool swap_inc = k >= 2 && !(o && o->swap_full);
  L->sg = take(swap_inc ? 8 * (size_t)n_pad * k_pad : 0);
  L->ss = take(swap_inc ? 8 * (size_t)n_pad : 0);
  L->gsym = take(8 * (size_t)n_pad);  // totals of the symmetric dense pass
  L->total = off;
  L->n_pad = n_pad;
  L->k_pad = k_pad;
  L->cap = cap;
  return true;
}

km_status ffail(km_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define FK(call)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return ffail(KM_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                                   \
  } while (0)

struct FCtx {
  FeatWs L;
  unsigned char* ws;
  FeatArgs a;
  cudaStream_t s;
  km_options opt;
  int sms;
  long long launches = 0;
  KmState* st() const { return reinterpret_cast<KmState*>(ws + L.st); }
};

km_status f_read(FCtx& c, KmState* h) {
  FK(cudaMemcpyAsync(h, c.st(), sizeof(KmState), cudaMemcpyDeviceToHost, c.s));
  FK(cudaStreamSynchronize(c.s));
  if (h->error) {
    char buf[256];
    const int e = state_message(*h, buf, sizeof(buf));
    return ffail((km_status)e, "%s", buf);
  }
  return KM_OK;
}

km_status f_reset(FCtx& c) {
  KmState h;
  memset(&h, 0, sizeof(h));
  h.last = -1;
  h.wait_ns = (unsigned long long)c.opt.wait_limit_ns;
  FK(cudaMemcpyAsync(c.st(), &h, sizeof(h), cudaMemcpyHostToDevice, c.s));
  return KM_OK;
}

km_status f_pass(FCtx& c, int mode, int first, cudaEvent_t ev0 = nullptr,
                 cudaEvent_t ev1 = nullptr) {
  FeatArgs a = c.a;
  a.mode = mode;
  a.build_first = first;
  const FeatLayout L = feat_layout(a.dk, a.k);
  if (L.total > 227 * 1024) return ffail(KM_E_UNSUPPORTED, "feature pass needs %zu B of shared memory", L.total);
  int grid = c.sms;
  if (grid > a.n_pad / kTileM) grid = a.n_pad / kTileM;
  if (grid > kFeatMaxGrid) grid = kFeatMaxGrid;
  if (mode == kModeSwap)
    FK(cudaFuncSetAttribute(k_feat_pass<kModeSwap>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  else if (mode == kModeBuild)
    FK(cudaFuncSetAttribute(k_feat_pass<kModeBuild>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  else if (mode == kModeBuildUpd)
    FK(cudaFuncSetAttribute(k_feat_pass<kModeBuildUpd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)L.total));
  else if (mode == kModeBuildSym)
    FK(cudaFuncSetAttribute(k_feat_pass<kModeBuildSym>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)L.total));
  else
    FK(cudaFuncSetAttribute(k_feat_pass<kModeSwapUpd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)L.total));
  // the symmetric pass adds into zeroed totals
  if (mode == kModeBuildSym) FK(cudaMemsetAsync(a.gsym, 0, 8 * (size_t)a.n_pad, c.s));
  if (ev0) FK(cudaEventRecord(ev0, c.s));
  if (mode == kModeSwap)
    k_feat_pass<kModeSwap><<<grid, kFeatThreads, L.total, c.s>>>(a);
  else if (mode == kModeBuild)
    k_feat_pass<kModeBuild><<<grid, kFeatThreads, L.total, c.s>>>(a);
  else if (mode == kModeBuildUpd)
    k_feat_pass<kModeBuildUpd><<<grid, kFeatThreads, L.total, c.s>>>(a);
  else if (mode == kModeBuildSym)
    k_feat_pass<kModeBuildSym><<<grid, kFeatThreads, L.total, c.s>>>(a);
  else
    k_feat_pass<kModeSwapUpd><<<grid, kFeatThreads, L.total, c.s>>>(a);
  FK(cudaGetLastError());
  if (ev1) FK(cudaEventRecord(ev1, c.s));
  ++c.launches;
  return KM_OK;
}

km_status f_cache(FCtx& c) {
  FK(cudaMemsetAsync(c.a.is_med, 0, (size_t)c.L.n_pad, c.s));
  if (c.a.swap_incremental) {
    FK(cudaMemsetAsync(c.a.lcnt, 0, 4, c.s));
    FK(cudaMemsetAsync(c.a.sg, 0, 8 * (size_t)c.L.n_pad * c.L.k_pad, c.s));
    FK(cudaMemsetAsync(c.a.ss, 0, 8 * (size_t)c.L.n_pad, c.s));
  }
  FK(cudaMemsetAsync(c.a.removal, 0, 16 * (size_t)c.L.k_pad, c.s));
  FK(cudaMemsetAsync(c.a.td2, 0, 16, c.s));
  k_feat_mark<<<(c.a.k + 255) / 256, 256, 0, c.s>>>(c.a);
  FK(cudaGetLastError());
  const size_t sm = 8 * (size_t)c.a.k;
  FK(cudaFuncSetAttribute(k_feat_cache, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_feat_cache<<<(c.L.n_pad + 255) / 256, 256, sm, c.s>>>(c.a);
  FK(cudaGetLastError());
  c.launches += 2;
  return KM_OK;
}

km_status run_features(bool do_build, bool do_swap, const void* X, int64_t n, int32_t d,
                       int64_t ldx, int32_t k, int32_t* medoids, int32_t* labels,
                       const km_options* opts, km_result* res, void* ws, size_t ws_bytes,
                       void* stream) {
  set_last_error("");
  if (!X || !medoids || !ws) return ffail(KM_E_INVALID, "NULL pointer");
  km_options def;
  km_default_options(&def);
  FCtx c;
  c.opt = opts ? *opts : def;
  if (c.opt.variant != KM_FASTPAM1)
    return ffail(KM_E_UNSUPPORTED, "the feature form implements FastPAM1 SWAP only");
  if (!feat_ws(n, d, k, &c.opt, &c.L))
    return ffail(KM_E_INVALID, "need 1 <= k <= n <= 2^28 and d a multiple of 16 up to %d",
                 kFeatMaxD - 16);
  if (k > kFeatMaxK) return ffail(KM_E_UNSUPPORTED, "feature form supports k <= %d", kFeatMaxK);
  if (ldx < d || ldx % 8) return ffail(KM_E_INVALID, "ldx must be >= d and a multiple of 8");
  if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(ws) % 256)
    return ffail(KM_E_INVALID, "X must be 16-byte and ws 256-byte aligned");
  if (ws_bytes < c.L.total)
    return ffail(KM_E_WORKSPACE, "workspace too small: %zu < %zu", ws_bytes, c.L.total);
  if (c.opt.wait_limit_ns < 0) return ffail(KM_E_INVALID, "wait_limit_ns must be >= 0");
  if (c.opt.max_iter <= 0) c.opt.max_iter = 100 * k + 100;
  c.ws = static_cast<unsigned char*>(ws);
  c.s = static_cast<cudaStream_t>(stream);
  c.sms = device_sm_count();
  if (c.sms <= 0) return ffail(KM_E_CUDA, "no CUDA device");
  FeatArgs& a = c.a;
  memset(&a, 0, sizeof(a));
  a.X = static_cast<const uint16_t*>(X);
  a.ldx = ldx;
  a.n = (int)n;
  a.d = d;
  a.k = k;
  a.n_pad = c.L.n_pad;
  a.k_pad = c.L.k_pad;
  a.dk = d + 16;
  a.XpA = reinterpret_cast<const uint16_t*>(c.ws + c.L.xpa);
  a.XpB = reinterpret_cast<uint16_t*>(c.ws + c.L.xpb);
  a.norms = reinterpret_cast<const float*>(c.ws + c.L.norms);
  a.near = reinterpret_cast<int32_t*>(c.ws + c.L.near);
  a.sec = reinterpret_cast<int32_t*>(c.ws + c.L.sec);
  a.dn = reinterpret_cast<float*>(c.ws + c.L.dn);
  a.ds = reinterpret_cast<float*>(c.ws + c.L.ds);
  a.dn2 = reinterpret_cast<float*>(c.ws + c.L.dn2);
  a.ds2 = reinterpret_cast<float*>(c.ws + c.L.ds2);
  a.thr = reinterpret_cast<float*>(c.ws + c.L.thr);
  a.is_med = c.ws + c.L.is_med;
  a.med = reinterpret_cast<int32_t*>(c.ws + c.L.med);
  a.removal = reinterpret_cast<long long*>(c.ws + c.L.removal);
  a.carry = reinterpret_cast<unsigned*>(c.ws + c.L.carry);
  a.range = reinterpret_cast<float*>(c.ws + c.L.range);
  a.td2 = reinterpret_cast<double*>(c.ws + c.L.td2);
  a.st = c.st();
  a.partials = c.ws + c.L.partials;
  a.gains = reinterpret_cast<double*>(c.ws + c.L.gains);
  a.trace = c.ws + c.L.trace;
  a.trace_cap = c.L.cap;
  a.tol = c.opt.tol;
  a.incremental = c.opt.build_full ? 0 : 1;
  a.XpL = reinterpret_cast<uint16_t*>(c.ws + c.L.xpl);
  a.lno = reinterpret_cast<float*>(c.ws + c.L.lno);
  a.lthr = reinterpret_cast<float*>(c.ws + c.L.lthr);
  a.lqo = reinterpret_cast<int*>(c.ws + c.L.lqo);
  a.lqn = reinterpret_cast<int*>(c.ws + c.L.lqn);
  a.lcnt = reinterpret_cast<unsigned*>(c.ws + c.L.lcnt);
  a.bgain = reinterpret_cast<long long*>(c.ws + c.L.bgain);
  a.swap_incremental = (k >= 2 && !c.opt.swap_full) ? 1 : 0;
  a.lnear = reinterpret_cast<int*>(c.ws + c.L.lnear);
  a.lqo2 = reinterpret_cast<int*>(c.ws + c.L.lno);  // the BUILD list is done by then
  a.lqn2 = reinterpret_cast<int*>(c.ws + c.L.lqn2);
  a.sg = reinterpret_cast<long long*>(c.ws + c.L.sg);
  a.ss = reinterpret_cast<long long*>(c.ws + c.L.ss);
  a.gsym = reinterpret_cast<unsigned long long*>(c.ws + c.L.gsym);
  if (res) memset(res, 0, sizeof(*res));

  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  const bool prof = c.opt.profile != 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> bev, sev;
  if (prof) {
    FK(cudaEventCreate(&e0));
    FK(cudaEventCreate(&e1));
    FK(cudaEventCreate(&e2));
  }
  km_status r = f_reset(c);
  if (r != KM_OK) return r;
  FK(launch_row_norms(X, ldx, (int)n, d, c.L.n_pad, const_cast<float*>(a.norms), c.s));
  {
    long long chunks = (long long)c.L.n_pad * (a.dk / 8);
    int grid = (int)((chunks + 255) / 256);
    if (grid > c.sms * 16) grid = c.sms * 16;
    k_feat_prearrange<<<grid, 256, 0, c.s>>>(a);
    FK(cudaGetLastError());
  }
  c.launches += 2;
  // fixed-point scale of the sums: q such that the diameter of the data's
  // bounding box (an upper bound of every distance) is below 2^25 units
  FK(cudaMemsetAsync(a.carry, 0, 4 * (size_t)kFeatMaxGrid * kTileM * c.L.k_pad, c.s));
  FK(cudaMemsetAsync(a.range, 0x7f, 4 * (size_t)d, c.s));
  FK(cudaMemsetAsync(a.range + d, 0x80, 4 * (size_t)d, c.s));
  k_feat_range<<<(int)(n < 2048 ? n : 2048), (d + 31) / 32 * 32, 0, c.s>>>(a);
  FK(cudaGetLastError());
  ++c.launches;
  {
    std::vector<int> rg(2 * (size_t)d);
    FK(cudaMemcpyAsync(rg.data(), a.range, 8 * (size_t)d, cudaMemcpyDeviceToHost, c.s));
    FK(cudaStreamSynchronize(c.s));
    double diam2 = 0.0;
    for (int t = 0; t < d; ++t) {
      int lo = rg[t], hi = rg[d + t];
      lo = lo >= 0 ? lo : lo ^ 0x7fffffff;
      hi = hi >= 0 ? hi : hi ^ 0x7fffffff;
      float flo, fhi;
      memcpy(&flo, &lo, 4);
      memcpy(&fhi, &hi, 4);
      const double w = (double)fhi - (double)flo;
      diam2 += w * w;
    }
    const double diam = std::sqrt(diam2) * (1.0 + 1.0 / 1024.0);
    int e = -126;
    if (diam > 0.0 && std::isfinite(diam)) (void)std::frexp(diam, &e);  // diam < 2^e
    int q = kFeatUnitBits - e;
    if (q > 40) q = 40;
    if (q < -100) q = -100;
    a.fq = q;
  }
  if (prof) FK(cudaEventRecord(e0, c.s));
  KmState h;
  memset(&h, 0, sizeof(h));
  if (do_build) {
    FK(cudaMemsetAsync(a.is_med, 0, (size_t)c.L.n_pad, c.s));
    if (a.incremental) {
      // rows of the list past its length are streamed but never counted;
      // zeros keep them finite
      FK(cudaMemsetAsync(a.XpL, 0, (size_t)c.L.n_pad * a.dk * 2, c.s));
      FK(cudaMemsetAsync(a.lcnt, 0, 16, c.s));
      FK(cudaMemsetAsync(a.bgain, 0, 8 * (size_t)c.L.n_pad, c.s));
    }
    for (int step = 0; step < k; ++step) {
      cudaEvent_t x0 = nullptr, x1 = nullptr;
      if (prof) {
        FK(cudaEventCreate(&x0));
        FK(cudaEventCreate(&x1));
        bev.push_back({x0, x1});
      }
      // step 0: every pair (each Gram tile pair once unless gram_full);
      // later steps: the listed points, or every candidate row again
      const int mode = (step == 0) ? (c.opt.gram_full ? kModeBuild : kModeBuildSym)
                                   : (a.incremental ? kModeBuildUpd : kModeBuild);
      r = f_pass(c, mode, step == 0, x0, x1);
      if (r != KM_OK) return r;
      FeatArgs b = a;
      b.build_first = (step == 0);
      k_feat_build_commit<<<(c.L.n_pad + 255) / 256, 256, 0, c.s>>>(b);
      FK(cudaGetLastError());
      ++c.launches;
    }
    r = f_read(c, &h);
    if (r != KM_OK) return r;
    if (res) {
      res->build_steps = h.build_step;
      res->td_initial = h.td_book_d;
      // point rows the BUILD passes streamed: every point in the dense step
      // 0 (and in every step of the plain pass), the lists after that
      unsigned long long upd = 0;
      if (a.incremental)
        FK(cudaMemcpy(&upd, reinterpret_cast<unsigned long long*>(a.lcnt) + 1, 8,
                      cudaMemcpyDeviceToHost));
      res->build_rows = a.incremental ? (long long)n + (long long)upd : (long long)n * k;
    }
    if (c.opt.build_gains)
      FK(cudaMemcpy(c.opt.build_gains, a.gains, 8 * (size_t)k, cudaMemcpyDeviceToHost));
  } else {
    FK(cudaMemcpyAsync(a.med, medoids, 4 * (size_t)k, cudaMemcpyDeviceToDevice, c.s));
  }
  if (prof) FK(cudaEventRecord(e1, c.s));
  km_status conv = KM_OK;
  r = f_reset(c);
  if (r != KM_OK) return r;
  r = f_cache(c);
  if (r != KM_OK) return r;
  if (do_swap && k == 1 && n > 1) {
    // k = 1: the best single swap is the 1-medoid (Eq. (3)); a dense pass
    // sums every non-medoid's distances, compared with the current TD
    KmState h0;
    r = f_read(c, &h0);
    if (r != KM_OK) return r;
    r = f_pass(c, c.opt.gram_full ? kModeBuild : kModeBuildSym, 1);
    if (r != KM_OK) return r;
    KmState h1;
    r = f_read(c, &h1);
    if (r != KM_OK) return r;
    int iters = 1, swaps = 0;
    if (h1.build_cand >= 0 && c.opt.max_iter >= 1 &&
        h1.build_gain_d - h0.td_book_d < -c.opt.tol) {
      const int cb = h1.build_cand;
      FK(cudaMemcpyAsync(a.med, &cb, 4, cudaMemcpyHostToDevice, c.s));
      if (c.L.cap > 0) {
        TraceRec t;
        memset(&t, 0, sizeof(t));
        t.d = h1.build_gain_d - h0.td_book_d;
        t.slot = 0;
        t.cand = cb;
        FK(cudaMemcpyAsync(a.trace, &t, sizeof(t), cudaMemcpyHostToDevice, c.s));
      }
      swaps = 1;
      iters = (c.opt.max_iter >= 2) ? 2 : 1;
    }
    r = f_reset(c);
    if (r != KM_OK) return r;
    r = f_cache(c);
    if (r != KM_OK) return r;
    h = KmState();
    r = f_read(c, &h);
    if (r != KM_OK) return r;
    // record the outcome in the state read back below
    KmState hs = h;
    hs.iter = iters;
    hs.swaps = swaps;
    hs.ntrace = swaps;
    hs.done = (swaps == 0 || c.opt.max_iter >= 2) ? 1 : 0;
    FK(cudaMemcpyAsync(c.st(), &hs, sizeof(hs), cudaMemcpyHostToDevice, c.s));
    if (!hs.done) conv = KM_E_NOT_CONVERGED;
  } else if (do_swap && k < n) {
    int launched = 0, batch = 1;
    const size_t sm = 8 * (size_t)k;
    FK(cudaFuncSetAttribute(k_feat_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    while (true) {
      int nb = batch;
      if (launched + nb > c.opt.max_iter) nb = c.opt.max_iter - launched;
      for (int j = 0; j < nb; ++j) {
        cudaEvent_t x0 = nullptr, x1 = nullptr;
        if (prof) {
          FK(cudaEventCreate(&x0));
          FK(cudaEventCreate(&x1));
          sev.push_back({x0, x1});
        }
        r = f_pass(c, a.swap_incremental ? kModeSwapUpd : kModeSwap, 0, x0, x1);
        if (r != KM_OK) return r;
        k_feat_apply<<<(a.n + 255) / 256, 256, sm, c.s>>>(a);
        FK(cudaGetLastError());
        ++c.launches;
      }
      launched += nb;
      r = f_read(c, &h);
      if (r != KM_OK) return r;
      if (h.done || launched >= c.opt.max_iter) break;
      batch = batch < 32 ? batch * 2 : 32;
    }
    if (!h.done) conv = KM_E_NOT_CONVERGED;
  }
  if (prof) FK(cudaEventRecord(e2, c.s));
  r = f_read(c, &h);
  if (r != KM_OK) return r;
  double td = 0.0;
  FK(cudaMemcpyAsync(&td, a.td2 + h.rb, 8, cudaMemcpyDeviceToHost, c.s));
  FK(cudaMemcpyAsync(medoids, a.med, 4 * (size_t)k, cudaMemcpyDeviceToDevice, c.s));
  if (labels) FK(cudaMemcpyAsync(labels, a.near, 4 * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  const int nt = h.ntrace < c.L.cap ? h.ntrace : c.L.cap;
  std::vector<TraceRec> tr((size_t)(nt > 0 ? nt : 0));
  if (nt > 0) FK(cudaMemcpyAsync(tr.data(), a.trace, sizeof(TraceRec) * nt, cudaMemcpyDeviceToHost, c.s));
  FK(cudaStreamSynchronize(c.s));
  for (int i = 0; i < nt; ++i) {
    if (c.opt.trace_delta) c.opt.trace_delta[i] = tr[i].d;
    if (c.opt.trace_slot) c.opt.trace_slot[i] = tr[i].slot;
    if (c.opt.trace_cand) c.opt.trace_cand[i] = tr[i].cand;
    if (c.opt.trace_time_ns) c.opt.trace_time_ns[i] = tr[i].t_ns;
  }
  if (res) {
    res->td = td;
    res->td_bookkept = h.td_book_d;
    res->iterations = h.iter;
    res->swaps = h.swaps;
    res->status = conv;
    res->kernel_launches = c.launches;
    if (prof) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      res->build_ms = ms;
      cudaEventElapsedTime(&ms, e1, e2);
      res->swap_ms = ms;
      double sb = 0.0, ss = 0.0;
      for (auto& p : bev) {
        cudaEventElapsedTime(&ms, p.first, p.second);
        sb += ms;
      }
      int cnt = 0;
      std::vector<double> per;
      for (auto& p : sev) {
        if (cnt >= h.iter) break;
        cudaEventElapsedTime(&ms, p.first, p.second);
        ss += ms;
        per.push_back(ms);
        ++cnt;
      }
      res->build_eval_ms = sb;
      res->build_launches = (int)bev.size();
      res->eval_ms = ss;
      res->eval_launches = cnt;
      if (!per.empty()) {
        res->eval_ms_first = per[0];
        std::sort(per.begin(), per.end());
        const size_t m = per.size() / 2;
        res->eval_ms_median = (per.size() % 2) ? per[m] : 0.5 * (per[m - 1] + per[m]);
      }
    }
  }
  if (prof) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    for (auto& p : bev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    for (auto& p : sev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
  }
  if (conv != KM_OK) ffail(conv, "max_iter reached before convergence");
  return conv;
}

}  // namespace

extern "C" size_t kmedoids_features_workspace_size(int64_t n, int32_t d, int32_t k,
                                                   const km_options* opts) {
  FeatWs L;
  km_options def;
  km_default_options(&def);
  if (!feat_ws(n, d, k, opts ? opts : &def, &L)) return 0;
  return L.total;
}

extern "C" km_status kmedoids_run_features(const void* X, int64_t n, int32_t d, int64_t ldx,
                                           int32_t k, int32_t* medoids_out, int32_t* labels_out,
                                           const km_options* opts, km_result* res, void* ws,
                                           size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_run_features");
  return run_features(true, true, X, n, d, ldx, k, medoids_out, labels_out, opts, res, ws,
                      ws_bytes, stream);
}

extern "C" km_status kmedoids_build_features(const void* X, int64_t n, int32_t d, int64_t ldx,
                                             int32_t k, int32_t* medoids_out, int32_t* labels_out,
                                             const km_options* opts, km_result* res, void* ws,
                                             size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_build_features");
  return run_features(true, false, X, n, d, ldx, k, medoids_out, labels_out, opts, res, ws,
                      ws_bytes, stream);
}

extern "C" km_status kmedoids_swap_features(const void* X, int64_t n, int32_t d, int64_t ldx,
                                            int32_t k, int32_t* medoids_inout,
                                            int32_t* labels_out, const km_options* opts,
                                            km_result* res, void* ws, size_t ws_bytes,
                                            void* stream) {
  NvtxRange nv("kmedoids_swap_features");
  return run_features(false, true, X, n, d, ldx, k, medoids_inout, labels_out, opts, res, ws,
                      ws_bytes, stream);
}

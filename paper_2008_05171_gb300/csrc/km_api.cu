// km_api.cu -- the C ABI of libkmedoids for the matrix form and its
// bichromatic variant (declared in include/kmedoids.h): argument checks,
// workspace carving and the enqueue of BUILD (Alg. 1) and SWAP (Alg. 3
// FastPAM1, Sec. 3.2 FastPAM2, Alg. 4 FasterPAM, Sec. 3.4 FastCLARANS),
// plus the initialisations of Sec. 3.3.  All arithmetic of the method runs
// in the kernels of km_stream.cu, km_points.cu, km_build.cu, km_eager.cu and
// km_init.cu; this file orders launches.  FastPAM1 without per-pass timing
// runs its loop as one cached CUDA graph (a conditional WHILE node) and a
// run reads its results once at the end; with per-pass timing and for
// FastPAM2 the host reads the device state record between batches of
// passes.
#define KM_SRC_ID 10  // names this file in bounds-check reports
#include <cmath>
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/kmedoids.h"
#include "km_device.cuh"
#include "km_internal.h"

using namespace km;

namespace {

thread_local std::string g_err;

km_status fail(km_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define KM_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(KM_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                  \
  } while (0)

// a kernel launch through a launcher returning cudaError_t, counted
#define KM_LAUNCH(ctx, call) \
  do {                       \
    KM_CUDA(call);           \
    ++(ctx).launches;        \
  } while (0)

size_t al(size_t x) { return (x + 255) / 256 * 256; }
int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct WsLayout {
  size_t st, med, is_med, near, sec, dn, ds, bdn, removal, td2, partials, slot_partials,
      slot_best, fp2_order, win_delta, win_slot, trace, gains, cand_gain, blist, blvn, blvo,
      baux, btt, bparts, blk, total;
  int64_t n_pad;  // points (columns), padded
  int64_t m_pad;  // candidate rows, padded (n_pad unless bichromatic)
  int k_pad;
  int trace_cap;
};

// m candidate rows (locations), n points (columns); m = n for the square
// matrix.
bool make_ws(int64_t m, int64_t n, int k, const km_options* o, WsLayout* L) {
  if (n <= 0 || m <= 0 || k <= 0 || k > m || n > (int64_t)INT32_MAX - 2 * kChunk ||
      m > (int64_t)INT32_MAX - 2 * kChunk)
    return false;
  const int64_t n_pad = rup(n, kChunk);
  const int64_t m_pad = rup(m, kChunk);
  const int k_pad = (int)rup(k, 32);
  const int variant = o ? o->variant : KM_FASTPAM1;
  const int cap = (o && o->trace_capacity > 0) ? o->trace_capacity : 0;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off += al(bytes);
    return r;
  };
  L->st = take(512);
  L->med = take(4 * (size_t)k_pad);
  L->is_med = take((size_t)m_pad);
  L->near = take(4 * (size_t)n_pad);
  L->sec = take(4 * (size_t)n_pad);
  L->dn = take(4 * (size_t)n_pad);
  L->ds = take(4 * (size_t)n_pad);
  L->bdn = take(4 * (size_t)n_pad);
  L->removal = take(8 * 2 * (size_t)k_pad);
  L->td2 = take(16);
  L->partials = take(16 * (size_t)kMaxGrid);
  L->slot_partials = take(variant == KM_FASTPAM2 ? 16 * (size_t)kMaxGrid * k : 0);
  L->slot_best = take(16 * (size_t)k);
  L->fp2_order = take(4 * (size_t)k);
  L->win_delta = take(8 * (size_t)kMaxGrid * kMaxRows);
  L->win_slot = take(4 * (size_t)kMaxGrid * kMaxRows);
  L->trace = take(sizeof(TraceRec) * (size_t)(cap > 0 ? cap : 1));
  L->gains = take(8 * (size_t)k);
  L->cand_gain = take(8 * (size_t)m_pad);  // also the incremental BUILD's gains
  L->blist = take(4 * (size_t)n_pad);
  L->blvn = take(4 * (size_t)n_pad);
  L->blvo = take(4 * (size_t)n_pad);
  L->baux = take(sizeof(BuildAux));
  L->btt = take(4 * (size_t)(n_pad / kChunk));
  L->bparts = take(16 * (size_t)(n_pad / kChunk));
  // results gathered for one read: the final state record, the record as
  // BUILD left it, the TD pair, the BUILD's row count and gains
  L->blk = take(1088 + 8 * (size_t)k_pad);
  L->total = off;
  L->n_pad = n_pad;
  L->m_pad = m_pad;
  L->k_pad = k_pad;
  L->trace_cap = cap;
  return true;
}

struct Ctx {
  const void* D;
  int dtype;
  int n;   // points (columns)
  int m;   // candidate rows (n unless bichromatic)
  long long ld;
  int k;
  unsigned char* ws;
  WsLayout L;
  cudaStream_t s;
  km_options opt;
  int sms;
  long long launches = 0;
  int fshift = 0;
  bool scanned = false;
  int swap_geom = 0, build_geom = 0;  // geometry table entries used
  long long build_rows = 0;           // rows the BUILD passes streamed (-1: on the device)
  bool graph_loop = false;            // the SWAP loop ran as one graph
  KmState* st() const { return reinterpret_cast<KmState*>(ws + L.st); }
  int esize() const { return dtype == KM_U16 ? 2 : 4; }  // bytes per matrix element
  template <class P>
  P* at(size_t off) const {
    return reinterpret_cast<P*>(ws + off);
  }
};

km_status check_common(const void* D, int32_t dtype, int64_t m, int64_t n, int64_t ld, int32_t k,
                       void* ws, size_t ws_bytes, const km_options* opts, Ctx* c) {
  if (!D) return fail(KM_E_INVALID, "D is NULL");
  if (dtype != KM_I32 && dtype != KM_F32 && dtype != KM_U16)
    return fail(KM_E_INVALID, "unknown dtype %d", dtype);
  if (n <= 0) return fail(KM_E_INVALID, "n must be positive (got %lld)", (long long)n);
  if (m <= 0) return fail(KM_E_INVALID, "m must be positive (got %lld)", (long long)m);
  if (n > (int64_t)INT32_MAX - 2 * kChunk || m > (int64_t)INT32_MAX - 2 * kChunk)
    return fail(KM_E_INVALID, "n too large");
  if (k < 1 || k > m) return fail(KM_E_INVALID, "need 1 <= k <= %s (k=%d, %lld)", m == n ? "n" : "m",
                                  k, (long long)m);
  if (ld < n) return fail(KM_E_INVALID, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
  if (ld % 4 != 0) return fail(KM_E_INVALID, "ld (%lld) must be a multiple of 4", (long long)ld);
  if (dtype == KM_U16 && ld % 8 != 0)
    return fail(KM_E_INVALID, "ld (%lld) must be a multiple of 8 for KM_U16", (long long)ld);
  if (reinterpret_cast<uintptr_t>(D) % 16 != 0) return fail(KM_E_INVALID, "D must be 16-byte aligned");
  if (!ws) return fail(KM_E_INVALID, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(KM_E_INVALID, "workspace must be 256-byte aligned");
  km_options def;
  km_default_options(&def);
  c->opt = opts ? *opts : def;
  if (c->opt.variant < 0 || c->opt.variant > 3) return fail(KM_E_INVALID, "unknown variant %d", c->opt.variant);
  if (c->opt.variant == KM_FASTCLARANS &&
      (!c->opt.draws || c->opt.draws_len < 1 || c->opt.maxneighbor < 1 || k < 2 || k >= m))
    return fail(KM_E_INVALID, "FastCLARANS needs draws, draws_len >= 1, maxneighbor >= 1 and "
                "2 <= k < n");
  if (!(c->opt.tol >= 0.0)) return fail(KM_E_INVALID, "tol must be >= 0");
  if (!(c->opt.fastpam2_tol >= 0.0)) return fail(KM_E_INVALID, "fastpam2_tol must be >= 0");
  if (c->opt.rows_per_tile != 0 && c->opt.rows_per_tile != 1 && c->opt.rows_per_tile != 2 &&
      c->opt.rows_per_tile != 4 && c->opt.rows_per_tile != 8 && c->opt.rows_per_tile != 16)
    return fail(KM_E_INVALID, "rows_per_tile must be 0, 1, 2, 4, 8 or 16");
  if (c->opt.trace_capacity < 0) return fail(KM_E_INVALID, "trace_capacity < 0");
  if (c->opt.tune < -1 || c->opt.tune > 16) return fail(KM_E_INVALID, "tune must be in -1..16");
  if (c->opt.wait_limit_ns < 0) return fail(KM_E_INVALID, "wait_limit_ns must be >= 0");
  if (!make_ws(m, n, k, &c->opt, &c->L)) return fail(KM_E_INVALID, "invalid sizes");
  if (ws_bytes < c->L.total)
    return fail(KM_E_WORKSPACE, "workspace too small: %zu < %zu bytes", ws_bytes, c->L.total);
  c->D = D;
  c->dtype = dtype;
  c->n = (int)n;
  c->m = (int)m;
  c->ld = ld;
  c->k = k;
  c->ws = static_cast<unsigned char*>(ws);
  c->sms = device_sm_count();
  if (c->sms <= 0) return fail(KM_E_CUDA, "no CUDA device");
  if (c->opt.max_iter <= 0) c->opt.max_iter = 100 * k + 100;
  return KM_OK;
}

StreamArgs stream_args(const Ctx& c) {
  StreamArgs a;
  memset(&a, 0, sizeof(a));
  a.D = c.D;
  a.ld = c.ld;
  a.n = c.n;
  a.m = c.m;
  a.k = c.k;
  a.k_pad = c.L.k_pad;
  a.n_pad = (int)c.L.n_pad;
  a.is_med = c.at<uint8_t>(c.L.is_med);
  a.dn = c.at<void>(c.L.dn);
  a.ds = c.at<void>(c.L.ds);
  a.near = c.at<int32_t>(c.L.near);
  a.bdn = c.at<void>(c.L.bdn);
  a.removal = c.at<void>(c.L.removal);
  a.td2 = c.at<void>(c.L.td2);
  a.st = c.st();
  a.partials = c.at<void>(c.L.partials);
  a.slot_partials = c.at<void>(c.L.slot_partials);
  a.slot_best = c.at<void>(c.L.slot_best);
  a.fp2_order = c.at<int32_t>(c.L.fp2_order);
  a.tol = c.opt.tol;
  a.fshift = c.fshift;
  return a;
}

PointArgs point_args(const Ctx& c) {
  PointArgs a;
  memset(&a, 0, sizeof(a));
  a.D = c.D;
  a.ld = c.ld;
  a.n = c.n;
  a.m = c.m;
  a.k = c.k;
  a.k_pad = c.L.k_pad;
  a.n_pad = (int)c.L.n_pad;
  a.med = c.at<int32_t>(c.L.med);
  a.is_med = c.at<uint8_t>(c.L.is_med);
  a.near = c.at<int32_t>(c.L.near);
  a.sec = c.at<int32_t>(c.L.sec);
  a.dn = c.at<void>(c.L.dn);
  a.ds = c.at<void>(c.L.ds);
  a.bdn = c.at<void>(c.L.bdn);
  a.removal = c.at<void>(c.L.removal);
  a.td2 = c.at<void>(c.L.td2);
  a.st = c.st();
  a.trace = c.at<void>(c.L.trace);
  a.trace_cap = c.L.trace_cap;
  a.partials = c.at<void>(c.L.partials);
  a.slot_best = c.at<void>(c.L.slot_best);
  a.fp2_order = c.at<int32_t>(c.L.fp2_order);
  a.gains = c.at<double>(c.L.gains);
  a.fp2_tol = c.opt.fastpam2_tol;
  a.fshift = c.fshift;
  a.scan = &c.st()->scan_max;
  return a;
}

int grid_for(const Ctx& c, const StreamConfig& cfg) {
  const int rows = cfg.rows;
  int g = c.sms * cfg.minb;
  const int need = (c.m + rows - 1) / rows;
  if (g > need) g = need;
  if (g > kMaxGrid) g = kMaxGrid;
  if (g < 1) g = 1;
  return g;
}

// Event pairs around kernel launches, summed after the final sync.
struct Timer {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  cudaStream_t s = nullptr;
  void start(bool enable, cudaStream_t st) {
    on = enable;
    s = st;
  }
  int mark() {  // returns event index or -1
    if (!on) return -1;
    if (used == ev.size()) {
      if (ev.size() >= 16384) return -1;
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      ev.push_back(e);
    }
    cudaEventRecord(ev[used], s);
    return (int)used++;
  }
  double ms(int a, int b) const {
    if (a < 0 || b < 0) return 0.0;
    float v = 0.f;
    cudaEventElapsedTime(&v, ev[a], ev[b]);
    return v;
  }
  ~Timer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

km_status state_error(const KmState& h);

km_status read_state(const Ctx& c, KmState* h) {
  KM_CUDA(cudaMemcpyAsync(h, c.st(), sizeof(KmState), cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  if (h->error) return state_error(*h);
  return KM_OK;
}

km_status reset_state(Ctx& c) {
  // on the device: a copy from pageable host memory would synchronise
  KM_LAUNCH(c, launch_reset_state(c.st(), (unsigned long long)c.opt.wait_limit_ns, c.s));
  return KM_OK;
}

// The message of a failure a kernel recorded in a state record.
km_status state_error(const KmState& h) {
  char buf[256];
  const int e = state_message(h, buf, sizeof(buf));
  return fail((km_status)e, "%s", buf);
}

// ------------------------------------------------------------- autotuning
// tune = -1: the first call for a (device, dtype, mode, variant, n, k) times
// one pass of every geometry of the table that fits, on the caller's own
// matrix and state, and keeps the fastest for the rest of the process.  The
// state record is restored before every timed pass, so the passes leave no
// trace; results do not depend on the geometry (exact sums, total orders).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, long long, int>, int> g_tune;

km_status config_for(Ctx& c, int mode, int flavour, const StreamArgs& sa, StreamConfig* cfg) {
  const char* what = (mode == kModeSwap) ? "SWAP" : "BUILD";
  if (c.opt.tune >= 0) {
    if (!stream_config(mode, c.k, flavour, c.opt.rows_per_tile, c.opt.tune, cfg, c.esize()))
      return fail(KM_E_UNSUPPORTED, "no %s kernel configuration fits (k=%d, tune=%d)", what, c.k,
                  c.opt.tune);
    return KM_OK;
  }
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, c.dtype, mode, flavour, (long long)c.n * (1ll << 31) + c.m,
                                   c.k * 64 + c.opt.rows_per_tile);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end() && stream_config(mode, c.k, flavour, 0, it->second, cfg, c.esize())) return KM_OK;
  }
  KmState saved;
  km_status r = read_state(c, &saved);
  if (r != KM_OK) return r;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KM_CUDA(cudaEventCreate(&e0));
  KM_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int g = 1; g <= 16; ++g) {
    StreamConfig cg;
    if (!stream_config(mode, c.k, flavour, 0, g, &cg, c.esize())) continue;
    if (c.opt.rows_per_tile > 0 && cg.rows != c.opt.rows_per_tile) continue;
    StreamArgs a = sa;
    a.win_rows = cg.rows;
    const int grid = grid_for(c, cg);
    float tmin = 0.f;
    for (int rep = 0; rep < 3; ++rep) {  // one warm-up, then the faster of two
      KM_CUDA(cudaMemcpyAsync(c.st(), &saved, sizeof(saved), cudaMemcpyHostToDevice, c.s));
      KM_CUDA(cudaEventRecord(e0, c.s));
      KM_LAUNCH(c, launch_stream(c.dtype, mode, cg, grid, a, c.s));
      KM_CUDA(cudaEventRecord(e1, c.s));
      KmState chk;
      r = read_state(c, &chk);  // synchronises; reports a device timeout
      if (r != KM_OK) break;
      float ms = 0.f;
      KM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1 || (rep == 2 && ms < tmin)) tmin = ms;
    }
    if (r != KM_OK) break;
    if (best == 0 || tmin < best_ms) {
      best = g;
      best_ms = tmin;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != KM_OK) return r;
  KM_CUDA(cudaMemcpyAsync(c.st(), &saved, sizeof(saved), cudaMemcpyHostToDevice, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  if (best == 0 || !stream_config(mode, c.k, flavour, 0, best, cfg, c.esize()))
    return fail(KM_E_UNSUPPORTED, "no %s kernel configuration fits (k=%d)", what, c.k);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return KM_OK;
}

// ------------------------------------------------------------------ BUILD
km_status scan_matrix(Ctx& c);

// The plain BUILD: every step streams all candidate rows (Alg. 1).
km_status do_build_full(Ctx& c, Timer& tm, std::vector<std::pair<int, int>>& ev, km_result* res) {
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.is_med), 0, (size_t)c.L.m_pad, c.s));
  StreamArgs sa = stream_args(c);
  sa.build_first = 1;
  StreamConfig cfg;
  km_status r = config_for(c, kModeBuild, 0, sa, &cfg);
  if (r != KM_OK) return r;
  c.build_geom = cfg.geometry;
  const int grid = grid_for(c, cfg);
  PointArgs pa = point_args(c);
  for (int step = 0; step < c.k; ++step) {
    sa.build_first = (step == 0);
    pa.build_first = (step == 0);
    const int e0 = tm.mark();
    KM_LAUNCH(c, launch_stream(c.dtype, kModeBuild, cfg, grid, sa, c.s));
    const int e1 = tm.mark();
    ev.push_back({e0, e1});
    KM_LAUNCH(c, launch_build_commit(c.dtype, pa, c.s));
  }
  if (res) res->build_launches = c.k;
  c.build_rows = 0;
  for (int t = 0; t < c.k; ++t) c.build_rows += c.m - t;
  return KM_OK;
}

BuildArgs build_args(const Ctx& c) {
  BuildArgs a;
  memset(&a, 0, sizeof(a));
  a.D = c.D;
  a.ld = c.ld;
  a.n = c.n;
  a.n_pad = (int)c.L.n_pad;
  a.k = c.k;
  a.fshift = c.fshift;
  a.st = c.st();
  a.aux = c.at<BuildAux>(c.L.baux);
  a.tticket = c.at<unsigned>(c.L.btt);
  a.partials = c.at<void>(c.L.bparts);
  a.cgain = c.at<long long>(c.L.cand_gain);
  a.list = c.at<int32_t>(c.L.blist);
  a.lvn = c.at<uint32_t>(c.L.blvn);
  a.lvo = c.at<uint32_t>(c.L.blvo);
  a.bdn = c.at<void>(c.L.bdn);
  a.med = c.at<int32_t>(c.L.med);
  a.is_med = c.at<uint8_t>(c.L.is_med);
  a.gains = c.at<double>(c.L.gains);
  return a;
}

// BUILD with incrementally updated gains (km_build.cu): step 0 sums every
// row, the gains after it take every row once more, and each later step
// streams only the rows of the points whose nearest distance the new medoid
// lowered.  Same choices as the plain pass in exact fixed point.
km_status do_build(Ctx& c, Timer& tm, std::vector<std::pair<int, int>>& ev, km_result* res) {
  NvtxRange nv("kmedoids BUILD");
  // the incremental gains read the rows of points as candidate columns
  // (symmetry): the bichromatic form takes the plain pass
  if (c.opt.build_full || c.m != c.n) return do_build_full(c, tm, ev, res);
  if (c.dtype == KM_F32 && !c.scanned) {
    km_status r = scan_matrix(c);  // fixed-point exponent of the gains
    if (r != KM_OK) return r;
    c.scanned = true;
  }
  const size_t tiles = (size_t)(c.L.n_pad / kChunk);
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.is_med), 0, (size_t)c.L.m_pad, c.s));
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.cand_gain), 0, 8 * (size_t)c.L.n_pad, c.s));
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.baux), 0, sizeof(BuildAux), c.s));
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.btt), 0, 4 * tiles, c.s));
  BuildArgs ba = build_args(c);
  const int groups = build_update_groups(c.n, c.sms);
  c.build_geom = 0;
  int e0 = tm.mark();
  KM_LAUNCH(c, launch_build_update(c.dtype, kBuildColsum, groups, ba, c.s));
  ev.push_back({e0, tm.mark()});
  for (int step = 0; step < c.k; ++step) {
    ba.first = (step == 0);
    ba.cur = step & 1;
    KM_LAUNCH(c, launch_build_add(c.dtype, ba, c.s));
    if (step + 1 < c.k) {
      e0 = tm.mark();
      KM_LAUNCH(c, launch_build_update(c.dtype, step == 0 ? kBuildFirst : kBuildStep, groups,
                                       ba, c.s));
      ev.push_back({e0, tm.mark()});
    }
  }
  if (res) res->build_launches = c.k;
  c.build_rows = -1;  // read back from the device after the BUILD
  return KM_OK;
}

// ------------------------------------------------------------------- SWAP
// Fixed-point exponent of the SWAP sums for float data: the largest entry M
// and n bound every sum a pass forms by 3 n M < 2^62.
km_status scan_matrix(Ctx& c) {
  if (c.dtype != KM_F32) {
    c.fshift = 0;
    return KM_OK;
  }
  PointArgs pa = point_args(c);
  KM_LAUNCH(c, launch_matrix_scan(pa, c.s));
  unsigned h[2] = {0, 0};
  KM_CUDA(cudaMemcpyAsync(h, &c.st()->scan_max, sizeof(h), cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  if (h[1]) return fail(KM_E_NUMERIC, "D holds a negative, infinite or NaN entry");
  float m;
  memcpy(&m, &h[0], 4);
  int em = 0;
  if (m > 0.f) (void)frexpf(m, &em);  // m < 2^em
  int bn = 0;
  while ((1ll << bn) <= (long long)c.n) ++bn;  // n < 2^bn
  c.fshift = 60 - bn - em;
  return KM_OK;
}

km_status swap_setup(Ctx& c) {
  if (c.dtype == KM_F32 && !c.scanned) {
    km_status r = scan_matrix(c);
    if (r != KM_OK) return r;
    c.scanned = true;
  }
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.is_med), 0, (size_t)c.L.m_pad, c.s));
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.removal), 0, 16 * (size_t)c.L.k_pad, c.s));
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.td2), 0, 16, c.s));
  PointArgs pa = point_args(c);
  KM_LAUNCH(c, launch_mark_medoids(pa, c.s));
  KM_LAUNCH(c, launch_cache_init(c.dtype, pa, c.s));
  return KM_OK;
}

km_status swap_k1(Ctx& c, KmState* h) {
  // k = 1: the best single swap is the 1-medoid (Eq. (3)); compare the
  // distance sums of every point with the current medoid's.
  StreamConfig cfg;
  if (!stream_config(kModeBuild, 1, 0, c.opt.rows_per_tile, c.opt.tune, &cfg, c.esize()))
    return fail(KM_E_UNSUPPORTED, "no kernel configuration fits");
  KM_CUDA(cudaMemsetAsync(c.at<void>(c.L.is_med), 0, (size_t)c.L.m_pad, c.s));
  StreamArgs sa = stream_args(c);
  sa.build_first = 1;
  sa.cand_gain = c.at<double>(c.L.cand_gain);
  KM_LAUNCH(c, launch_stream(c.dtype, kModeBuild, cfg, grid_for(c, cfg), sa, c.s));
  int32_t m = 0;
  KM_CUDA(cudaMemcpyAsync(&m, c.at<int32_t>(c.L.med), 4, cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  double sm = 0.0;
  KM_CUDA(cudaMemcpyAsync(&sm, c.at<double>(c.L.cand_gain) + m, 8, cudaMemcpyDeviceToHost, c.s));
  km_status e = read_state(c, h);
  if (e != KM_OK) return e;
  const double best = h->build_gain_d;
  const int cb = h->build_cand;
  int iters = 1, swaps = 0;
  if (cb != m && cb >= 0 && best - sm < -c.opt.tol && c.opt.max_iter >= 1) {
    KM_CUDA(cudaMemcpyAsync(c.at<int32_t>(c.L.med), &cb, 4, cudaMemcpyHostToDevice, c.s));
    swaps = 1;
    iters = (c.opt.max_iter >= 2) ? 2 : 1;
    if (c.L.trace_cap > 0) {
      TraceRec tr;
      memset(&tr, 0, sizeof(tr));
      tr.d = best - sm;
      tr.di = (long long)(best - sm);
      tr.slot = 0;
      tr.cand = cb;
      KM_CUDA(cudaMemcpyAsync(c.at<TraceRec>(c.L.trace), &tr, sizeof(tr), cudaMemcpyHostToDevice, c.s));
    }
  }
  KM_CUDA(cudaStreamSynchronize(c.s));
  // fresh state + cache for labels and the exact TD
  km_status r = reset_state(c);
  if (r != KM_OK) return r;
  r = swap_setup(c);
  if (r != KM_OK) return r;
  r = read_state(c, h);
  if (r != KM_OK) return r;
  h->iter = iters;
  h->swaps = swaps;
  h->ntrace = swaps;
  h->done = (swaps == 0 || c.opt.max_iter >= 2) ? 1 : 0;
  return KM_OK;
}

// ------------------------------------------------- SWAP loop as a graph
// FastPAM1 to convergence as one CUDA graph: a conditional WHILE node whose
// body is the evaluation pass, the swap and k_swap_loop_cond (which sets the
// condition from the device state record).  Built once per distinct set of
// kernel arguments (matrix, workspace, sizes, geometry, options) and kept,
// so a repeated call launches one graph and reads nothing back until the end.
struct SwapGraph {
  std::vector<unsigned char> key;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
};
std::mutex g_graph_mu;
std::vector<SwapGraph> g_graphs;  // most recently used last
constexpr size_t kMaxGraphs = 8;
std::map<int, cudaStream_t> g_cap_stream;  // per device, for capturing the loop bodies

template <class X>
void key_add(std::vector<unsigned char>& k, const X& x) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&x);
  k.insert(k.end(), p, p + sizeof(X));
}

// Launches the loop graph on c.s; *used = false (nothing enqueued) when a
// graph cannot be built here, so the caller runs the host-driven loop.
km_status swap_loop_graph(Ctx& c, const StreamConfig& cfg, int grid, const StreamArgs& sa,
                          const PointArgs& pa, bool* used) {
  *used = false;
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  std::vector<unsigned char> key;
  key_add(key, dev);
  key_add(key, c.dtype);
  key_add(key, cfg);
  key_add(key, grid);
  key_add(key, c.opt.max_iter);
  key_add(key, sa);
  key_add(key, pa);
  std::lock_guard<std::mutex> lk(g_graph_mu);
  cudaGraphExec_t exec = nullptr;
  for (size_t i = 0; i < g_graphs.size(); ++i)
    if (g_graphs[i].key == key) {
      SwapGraph e = g_graphs[i];
      g_graphs.erase(g_graphs.begin() + (long)i);
      g_graphs.push_back(e);
      exec = e.e;
      break;
    }
  if (!exec) {
    cudaStream_t cs = nullptr;
    auto it = g_cap_stream.find(dev);
    if (it != g_cap_stream.end()) {
      cs = it->second;
    } else {
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return KM_OK;
      g_cap_stream[dev] = cs;
    }
    SwapGraph ng;
    ng.key = key;
    bool ok = cudaGraphCreate(&ng.g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    memset(static_cast<void*>(&p), 0, sizeof(p));  // every union byte, ctx included
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, ng.g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = h;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      cudaGraphNode_t node;
      ok = cudaGraphAddNode(&node, ng.g, nullptr, nullptr, 0, &p) == cudaSuccess;
    }
    if (ok) {
      cudaGraph_t body = p.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed) == cudaSuccess;
      if (ok) {
        bool lok = launch_stream(c.dtype, kModeSwap, cfg, grid, sa, cs) == cudaSuccess;
        lok = lok && launch_apply(c.dtype, pa, cs) == cudaSuccess;
        lok = lok && launch_swap_loop_cond(c.st(), (unsigned long long)h, c.opt.max_iter, cs) ==
                         cudaSuccess;
        cudaGraph_t out = nullptr;
        const bool eok = cudaStreamEndCapture(cs, &out) == cudaSuccess;
        ok = lok && eok;
      }
    }
    if (ok) ok = cudaGraphInstantiate(&ng.e, ng.g, 0) == cudaSuccess;
    if (!ok) {
      if (ng.e) cudaGraphExecDestroy(ng.e);
      if (ng.g) cudaGraphDestroy(ng.g);
      (void)cudaGetLastError();  // the host-driven loop runs instead
      return KM_OK;
    }
    if (g_graphs.size() >= kMaxGraphs) {
      cudaGraphExecDestroy(g_graphs.front().e);
      cudaGraphDestroy(g_graphs.front().g);
      g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(ng);
    exec = ng.e;
  }
  KM_CUDA(cudaGraphLaunch(exec, c.s));
  *used = true;
  return KM_OK;
}

km_status do_swap(Ctx& c, Timer& tm, std::vector<std::pair<int, int>>& ev, KmState* h,
                  km_result* res) {
  NvtxRange nv("kmedoids SWAP");
  km_status r = swap_setup(c);
  if (r != KM_OK) return r;
  if (c.k == 1) return swap_k1(c, h);
  const int variant = c.opt.variant;
  const int flavour = variant == KM_FASTPAM2     ? kFastPAM2
                      : variant == KM_FASTERPAM   ? kFasterPAM
                      : variant == KM_FASTCLARANS ? kCLARANS
                                                  : kFastPAM1;
  StreamArgs sa = stream_args(c);
  sa.flavour = flavour;
  if (flavour == kFasterPAM || flavour == kCLARANS) {  // per-position window results
    sa.cand_delta = c.at<double>(c.L.win_delta);
    sa.cand_slot = c.at<int32_t>(c.L.win_slot);
  }
  if (flavour == kCLARANS) {
    sa.draws = c.opt.draws;
    sa.draws_len = c.opt.draws_len;
    sa.maxneighbor = c.opt.maxneighbor;
  }
  if ((flavour == kFasterPAM || flavour == kCLARANS) && c.opt.tune <= 0 && c.m == c.n) {
    // the eager variants run as one persistent cooperative launch when every
    // CTA of its grid can be resident (the usual case); a fixed geometry
    // (tune > 0) selects the windowed streaming kernel instead
    const int eg = eager_grid(c.dtype, c.k);
    const int rows = c.opt.rows_per_tile > 0 ? c.opt.rows_per_tile : 8;
    const long long cap = (long long)kMaxGrid * kMaxRows / 2;
    if (eg > 0 && (long long)eg * rows <= cap) {
      EagerArgs ea;
      memset(&ea, 0, sizeof(ea));
      ea.D = c.D;
      ea.ld = c.ld;
      ea.n = c.n;
      ea.k = c.k;
      ea.k_pad = c.L.k_pad;
      ea.fshift = c.fshift;
      ea.med = c.at<int32_t>(c.L.med);
      ea.is_med = c.at<uint8_t>(c.L.is_med);
      ea.near = c.at<int32_t>(c.L.near);
      ea.sec = c.at<int32_t>(c.L.sec);
      ea.dn = c.at<void>(c.L.dn);
      ea.ds = c.at<void>(c.L.ds);
      ea.removal = c.at<void>(c.L.removal);
      ea.td2 = c.at<void>(c.L.td2);
      ea.st = c.st();
      ea.win_delta = c.at<double>(c.L.win_delta);
      ea.win_slot = c.at<int32_t>(c.L.win_slot);
      ea.win_cap = cap;
      ea.win_rows = rows;
      ea.bar = c.st()->bar;
      ea.trace = c.at<void>(c.L.trace);
      ea.trace_cap = c.L.trace_cap;
      ea.flavour = flavour;
      ea.draws = c.opt.draws;
      ea.draws_len = c.opt.draws_len;
      ea.maxneighbor = c.opt.maxneighbor;
      ea.max_pos = (long long)c.opt.max_iter * c.n;
      ea.tol = c.opt.tol;
      c.swap_geom = 0;
      const int e0 = tm.mark();
      KM_LAUNCH(c, launch_eager(c.dtype, eg, ea, c.s));
      const int e1 = tm.mark();
      ev.push_back({e0, e1});
      return KM_OK;  // the caller reads the state once at the end
    }
  }
  StreamConfig cfg;
  r = config_for(c, kModeSwap, flavour, sa, &cfg);
  if (r != KM_OK) return r;
  c.swap_geom = cfg.geometry;
  sa.win_rows = cfg.rows;
  const int grid = grid_for(c, cfg);
  PointArgs pa = point_args(c);
  const int max_iter = c.opt.max_iter;

  if (variant == KM_FASTPAM1 && !tm.on) {
    // the whole loop on the device, one graph launch (per-pass event timing
    // with profile != 0 takes the host-driven loop below)
    bool used = false;
    km_status gr = swap_loop_graph(c, cfg, grid, sa, pa, &used);
    if (gr != KM_OK) return gr;
    if (used) {
      c.graph_loop = true;
      return KM_OK;
    }
  }
  if (variant == KM_FASTPAM1 || variant == KM_FASTERPAM || variant == KM_FASTCLARANS) {
    const long long pos_limit = (long long)max_iter * c.m;
    int launched = 0, batch = 1;
    const int max_launch = (variant == KM_FASTPAM1) ? max_iter : INT32_MAX;
    while (true) {
      int nb = batch;
      if (variant == KM_FASTPAM1 && launched + nb > max_launch) nb = max_launch - launched;
      for (int j = 0; j < nb; ++j) {
        const int e0 = tm.mark();
        KM_LAUNCH(c, launch_stream(c.dtype, kModeSwap, cfg, grid, sa, c.s));
        const int e1 = tm.mark();
        ev.push_back({e0, e1});
        KM_LAUNCH(c, launch_apply(c.dtype, pa, c.s));
      }
      launched += nb;
      r = read_state(c, h);
      if (r != KM_OK) return r;
      if (h->done) break;
      if (variant == KM_FASTPAM1 && launched >= max_launch) break;
      if (variant == KM_FASTERPAM && h->pos >= pos_limit) break;
      batch = batch < 64 ? batch * 2 : 64;
    }
  } else {
    // FastPAM2: evaluation pass, best swap, then the queued per-slot swaps
    while (h->iter < max_iter) {
      const int e0 = tm.mark();
      KM_LAUNCH(c, launch_stream(c.dtype, kModeSwap, cfg, grid, sa, c.s));
      const int e1 = tm.mark();
      ev.push_back({e0, e1});
      r = read_state(c, h);
      if (r != KM_OK) return r;
      if (h->done) break;
      KM_LAUNCH(c, launch_apply(c.dtype, pa, c.s));
      const int extra = h->fp2_extra;
      for (int q = 0; q < extra; ++q) {
        pa.fp2_index = q;
        KM_LAUNCH(c, launch_fp2_try(c.dtype, pa, c.s));
        KM_LAUNCH(c, launch_apply(c.dtype, pa, c.s));
      }
      r = read_state(c, h);
      if (r != KM_OK) return r;
    }
  }
  (void)res;
  return KM_OK;
}

// ------------------------------------------------------------- results
// Everything a call reports is gathered into the workspace's result block
// and read with one device-to-host copy, the call's one synchronisation
// (the trace, when one is asked for, follows in a second copy).
constexpr size_t kBlkFinal = 0, kBlkBuild = 512, kBlkTd = 1024, kBlkRows = 1040, kBlkGains = 1088;

struct Outcome {
  KmState fin;    // the state record at the end
  KmState bld;    // as BUILD left it
  double td_d = 0.0;
  long long td_i = 0;
  unsigned long long rows = 0;
};

km_status gather_and_read(Ctx& c, bool with_build, int32_t* medoids_out, int32_t* labels_out,
                          Outcome* o) {
  unsigned char* blk = c.ws + c.L.blk;
  if (medoids_out)
    KM_CUDA(cudaMemcpyAsync(medoids_out, c.at<int32_t>(c.L.med), 4 * (size_t)c.k,
                            cudaMemcpyDeviceToDevice, c.s));
  if (labels_out)
    KM_CUDA(cudaMemcpyAsync(labels_out, c.at<int32_t>(c.L.near), 4 * (size_t)c.n,
                            cudaMemcpyDeviceToDevice, c.s));
  KM_CUDA(cudaMemcpyAsync(blk + kBlkFinal, c.st(), sizeof(KmState), cudaMemcpyDeviceToDevice, c.s));
  KM_CUDA(cudaMemcpyAsync(blk + kBlkTd, c.at<void>(c.L.td2), 16, cudaMemcpyDeviceToDevice, c.s));
  size_t bytes = kBlkTd + 16;
  if (with_build) {
    KM_CUDA(cudaMemcpyAsync(blk + kBlkRows, &c.at<BuildAux>(c.L.baux)->rows_total, 8,
                            cudaMemcpyDeviceToDevice, c.s));
    bytes = kBlkRows + 8;
    if (c.opt.build_gains) {
      KM_CUDA(cudaMemcpyAsync(blk + kBlkGains, c.at<double>(c.L.gains), 8 * (size_t)c.k,
                              cudaMemcpyDeviceToDevice, c.s));
      bytes = kBlkGains + 8 * (size_t)c.k;
    }
  }
  std::vector<unsigned char> h(bytes);
  KM_CUDA(cudaMemcpyAsync(h.data(), blk, bytes, cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  memcpy(&o->fin, h.data() + kBlkFinal, sizeof(KmState));
  memset(&o->bld, 0, sizeof(KmState));
  if (with_build) {
    memcpy(&o->bld, h.data() + kBlkBuild, sizeof(KmState));
    memcpy(&o->rows, h.data() + kBlkRows, 8);
    if (o->bld.error) return state_error(o->bld);
  }
  if (o->fin.error) return state_error(o->fin);
  const int rb = o->fin.rb & 1;
  if (c.dtype != KM_F32)
    memcpy(&o->td_i, h.data() + kBlkTd + 8 * rb, 8);
  else
    memcpy(&o->td_d, h.data() + kBlkTd + 8 * rb, 8);
  if (with_build && c.opt.build_gains)
    memcpy(c.opt.build_gains, h.data() + kBlkGains, 8 * (size_t)c.k);
  return KM_OK;
}

km_status copy_trace(Ctx& c, int ntrace) {
  const int nt = ntrace < c.L.trace_cap ? ntrace : c.L.trace_cap;
  if (nt <= 0) return KM_OK;
  if (!c.opt.trace_delta && !c.opt.trace_slot && !c.opt.trace_cand && !c.opt.trace_time_ns)
    return KM_OK;
  std::vector<TraceRec> tr((size_t)nt);
  KM_CUDA(cudaMemcpyAsync(tr.data(), c.at<TraceRec>(c.L.trace), sizeof(TraceRec) * nt,
                          cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  for (int i = 0; i < nt; ++i) {
    if (c.opt.trace_delta) c.opt.trace_delta[i] = (c.dtype != KM_F32) ? (double)tr[i].di : tr[i].d;
    if (c.opt.trace_slot) c.opt.trace_slot[i] = tr[i].slot;
    if (c.opt.trace_cand) c.opt.trace_cand[i] = tr[i].cand;
    if (c.opt.trace_time_ns) c.opt.trace_time_ns[i] = tr[i].t_ns;
  }
  return KM_OK;
}

void eval_times(const Timer& tm, const std::vector<std::pair<int, int>>& ev_swap, int passes,
                km_result* res) {
  if (!tm.on || !res) return;
  double sum = 0.0;
  std::vector<double> per;
  for (auto& p : ev_swap) {
    if ((int)per.size() >= passes) break;
    const double v = tm.ms(p.first, p.second);
    sum += v;
    per.push_back(v);
  }
  res->eval_ms = sum;
  res->eval_launches = (int)per.size();
  if (!per.empty()) {
    res->eval_ms_first = per[0];
    std::sort(per.begin(), per.end());
    const size_t m = per.size() / 2;
    res->eval_ms_median = (per.size() % 2) ? per[m] : 0.5 * (per[m - 1] + per[m]);
  }
}

}  // namespace

void km::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

// ====================================================================== ABI
extern "C" {

void km_default_options(km_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->variant = KM_FASTPAM1;
  o->max_iter = 0;
  o->tol = 0.0;
  o->fastpam2_tol = 0.0;
}

size_t kmedoids_workspace_size(int64_t n, int32_t k, int32_t dtype, const km_options* opts) {
  if (dtype != KM_I32 && dtype != KM_F32 && dtype != KM_U16) return 0;
  WsLayout L;
  km_options def;
  km_default_options(&def);
  if (!make_ws(n, n, k, opts ? opts : &def, &L)) return 0;
  return L.total;
}

const char* kmedoids_last_error(void) { return g_err.c_str(); }

const char* kmedoids_version(void) { return "kmedoids-gb300 0.1 (sm_103a)"; }

static km_status run_impl(bool do_b, bool do_s, const void* D, int32_t dtype, int64_t m, int64_t n,
                          int64_t ld,
                          int32_t k, int32_t* medoids_io, int32_t* labels_out,
                          const km_options* opts, km_result* res, void* ws, size_t ws_bytes,
                          void* stream) {
  g_err.clear();
  NvtxRange nv(do_b ? (do_s ? "kmedoids_run" : "kmedoids_build") : "kmedoids_swap");
  Ctx c;
  km_status r = check_common(D, dtype, m, n, ld, k, ws, ws_bytes, opts, &c);
  if (r != KM_OK) {
    if (res) res->status = r;
    return r;
  }
  if (!medoids_io) return fail(KM_E_INVALID, "medoids pointer is NULL");
  if (m != n && c.opt.check_input)
    return fail(KM_E_INVALID, "check_input tests a square symmetric matrix (m = n)");
  c.s = static_cast<cudaStream_t>(stream);
  if (res) {
    memset(res, 0, sizeof(*res));
  }
  Timer tm;
  tm.start(c.opt.profile != 0, c.s);
  std::vector<std::pair<int, int>> ev_build, ev_swap;
  r = reset_state(c);
  if (r != KM_OK) return r;
  if (c.opt.check_input) {
    KM_LAUNCH(c, launch_matrix_check(c.dtype, c.D, c.ld, c.n, &c.st()->check_flags, c.s));
    unsigned fl = 0;
    KM_CUDA(cudaMemcpyAsync(&fl, &c.st()->check_flags, 4, cudaMemcpyDeviceToHost, c.s));
    KM_CUDA(cudaStreamSynchronize(c.s));
    if (fl & 4u) return fail(KM_E_NUMERIC, "D holds a negative, infinite or NaN entry");
    if (fl & 2u) return fail(KM_E_INVALID, "D has a nonzero diagonal entry");
    if (fl & 1u) return fail(KM_E_INVALID, "D is not symmetric");
  }
  KmState h;
  memset(&h, 0, sizeof(h));

  if (!do_b) {
    // validate the given medoids: in range and distinct
    std::vector<int32_t> hm((size_t)k);
    KM_CUDA(cudaMemcpyAsync(hm.data(), medoids_io, 4 * (size_t)k, cudaMemcpyDeviceToHost, c.s));
    KM_CUDA(cudaStreamSynchronize(c.s));
    std::vector<char> seen((size_t)m, 0);
    for (int j = 0; j < k; ++j) {
      if (hm[j] < 0 || hm[j] >= m) return fail(KM_E_INVALID, "medoid %d out of range: %d", j, hm[j]);
      if (seen[hm[j]]) return fail(KM_E_INVALID, "medoid %d repeated: %d", j, hm[j]);
      seen[hm[j]] = 1;
    }
    KM_CUDA(cudaMemcpyAsync(c.at<int32_t>(c.L.med), medoids_io, 4 * (size_t)k,
                            cudaMemcpyDeviceToDevice, c.s));
  }
  const int b0 = tm.mark();
  if (do_b) {
    r = do_build(c, tm, ev_build, res);
    if (r != KM_OK) return r;
  }
  const int b1 = tm.mark();
  KmState* st_build = reinterpret_cast<KmState*>(c.ws + c.L.blk + kBlkBuild);
  if (do_b && do_s)  // the SWAP resets the record: keep the BUILD's
    KM_LAUNCH(c, launch_build_handoff(c.st(), st_build, c.at<int32_t>(c.L.med), c.k, c.s));
  int s0 = -1, s1 = -1;
  if (do_s) {
    r = reset_state(c);
    if (r != KM_OK) return r;
    s0 = tm.mark();
    r = do_swap(c, tm, ev_swap, &h, res);
    s1 = tm.mark();
    if (r != KM_OK) {
      if (res) res->status = r;
      return r;
    }
  } else {
    // BUILD only: the cache of the result gives labels and the exact TD
    if (do_b)
      KM_CUDA(cudaMemcpyAsync(st_build, c.st(), sizeof(KmState), cudaMemcpyDeviceToDevice, c.s));
    r = reset_state(c);
    if (r != KM_OK) return r;
    r = swap_setup(c);
    if (r != KM_OK) return r;
  }
  Outcome o;
  r = gather_and_read(c, do_b, medoids_io, labels_out, &o);
  if (r != KM_OK) {
    if (res) res->status = r;
    return r;
  }
  KmState hf = o.fin;
  if (!do_s) {
    hf.iter = 0;
    hf.swaps = 0;
    hf.ntrace = 0;
    hf.done = 1;
  } else if (c.k == 1) {
    hf.iter = h.iter;
    hf.swaps = h.swaps;
    hf.ntrace = h.ntrace;
    hf.done = h.done;
  }
  if (c.graph_loop) c.launches += 3 * (long long)o.fin.loop_guard;
  r = copy_trace(c, hf.ntrace);
  if (r != KM_OK) return r;
  km_status conv = KM_OK;
  if (do_s) {
    if (!hf.done) conv = KM_E_NOT_CONVERGED;
    if (c.opt.variant == KM_FASTCLARANS && hf.fails < c.opt.maxneighbor) conv = KM_E_NOT_CONVERGED;
  }
  if (res) {
    res->td = (c.dtype != KM_F32) ? (double)o.td_i : o.td_d;
    res->td_i64 = (c.dtype != KM_F32) ? o.td_i : 0;
    res->td_bookkept = (c.dtype != KM_F32) ? (double)hf.td_book_i : hf.td_book_d;
    if (do_b) {
      res->build_steps = o.bld.build_step;
      res->build_rows = c.build_rows < 0 ? (long long)o.rows : c.build_rows;
      res->td_initial = (c.dtype != KM_F32) ? (double)o.bld.td_book_i : o.bld.td_book_d;
    }
    if (do_s) {
      res->iterations = hf.iter;
      res->swaps = hf.swaps;
      if (c.opt.variant == KM_FASTERPAM && c.k > 1) {
        res->visited = hf.pos;
        res->iterations = (int)((hf.pos + c.m - 1) / c.m);
      }
      if (c.opt.variant == KM_FASTCLARANS) {
        res->visited = hf.pos;
        res->iterations = (int)hf.evaluated;
      }
      if (c.opt.variant == KM_FASTERPAM || c.opt.variant == KM_FASTCLARANS)
        res->evaluated = hf.evaluated;
    }
    if (tm.on) {
      if (do_s) res->swap_ms = tm.ms(s0, s1);
      eval_times(tm, ev_swap, hf.iter, res);
      res->build_ms = tm.ms(b0, b1);
      double sb = 0.0;
      for (auto& p : ev_build) sb += tm.ms(p.first, p.second);
      res->build_eval_ms = sb;
    }
    res->status = conv;
    res->kernel_launches = c.launches;
    res->swap_geometry = (int16_t)c.swap_geom;
    res->build_geometry = (int16_t)c.build_geom;
  }
  if (conv != KM_OK) {
    if (c.opt.variant == KM_FASTCLARANS)
      fail(conv, "the %lld draws ran out before %lld consecutive failures",
           (long long)c.opt.draws_len, (long long)c.opt.maxneighbor);
    else
      fail(conv, "max_iter (%d) reached before convergence", c.opt.max_iter);
  }
  return conv;
}

km_status kmedoids_build(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                         int32_t* medoids_out, const km_options* opts, km_result* res, void* ws,
                         size_t ws_bytes, void* stream) {
  return run_impl(true, false, D, dtype, n, n, ld, k, medoids_out, nullptr, opts, res, ws, ws_bytes,
                  stream);
}

km_status kmedoids_swap(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                        int32_t* medoids_inout, int32_t* labels_out, const km_options* opts,
                        km_result* res, void* ws, size_t ws_bytes, void* stream) {
  return run_impl(false, true, D, dtype, n, n, ld, k, medoids_inout, labels_out, opts, res, ws,
                  ws_bytes, stream);
}

km_status kmedoids_run(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                       int32_t* medoids_out, int32_t* labels_out, const km_options* opts,
                       km_result* res, void* ws, size_t ws_bytes, void* stream) {
  return run_impl(true, true, D, dtype, n, n, ld, k, medoids_out, labels_out, opts, res, ws, ws_bytes,
                  stream);
}

size_t kmedoids_bichromatic_workspace_size(int64_t m, int64_t n, int32_t k, int32_t dtype,
                                           const km_options* opts) {
  if (dtype != KM_I32 && dtype != KM_F32 && dtype != KM_U16) return 0;
  WsLayout L;
  km_options def;
  km_default_options(&def);
  if (!make_ws(m, n, k, opts ? opts : &def, &L)) return 0;
  return L.total;
}

km_status kmedoids_run_bichromatic(const void* D, int32_t dtype, int64_t m, int64_t n, int64_t ld,
                                   int32_t k, int32_t* medoids_out, int32_t* labels_out,
                                   const km_options* opts, km_result* res, void* ws,
                                   size_t ws_bytes, void* stream) {
  return run_impl(true, true, D, dtype, m, n, ld, k, medoids_out, labels_out, opts, res, ws,
                  ws_bytes, stream);
}

km_status kmedoids_swap_bichromatic(const void* D, int32_t dtype, int64_t m, int64_t n,
                                    int64_t ld, int32_t k, int32_t* medoids_inout,
                                    int32_t* labels_out, const km_options* opts, km_result* res,
                                    void* ws, size_t ws_bytes, void* stream) {
  return run_impl(false, true, D, dtype, m, n, ld, k, medoids_inout, labels_out, opts, res, ws,
                  ws_bytes, stream);
}

km_status kmedoids_eval_swaps(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                              const int32_t* medoids, double* cand_delta, int32_t* cand_slot,
                              double* best_delta, int32_t* best_slot, int32_t* best_cand,
                              void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  Ctx c;
  km_status r = check_common(D, dtype, n, n, ld, k, ws, ws_bytes, nullptr, &c);
  if (r != KM_OK) return r;
  if (k < 2) return fail(KM_E_INVALID, "kmedoids_eval_swaps needs k >= 2");
  if (!medoids) return fail(KM_E_INVALID, "medoids is NULL");
  c.s = static_cast<cudaStream_t>(stream);
  r = reset_state(c);
  if (r != KM_OK) return r;
  KM_CUDA(cudaMemcpyAsync(c.at<int32_t>(c.L.med), medoids, 4 * (size_t)k, cudaMemcpyDeviceToDevice, c.s));
  r = swap_setup(c);
  if (r != KM_OK) return r;
  StreamConfig cfg;
  if (!stream_config(kModeSwap, k, kEvalOnly, 0, 0, &cfg, c.esize()))
    return fail(KM_E_UNSUPPORTED, "k=%d too large for the SWAP kernel", k);
  StreamArgs sa = stream_args(c);
  sa.flavour = kEvalOnly;
  sa.cand_delta = cand_delta;
  sa.cand_slot = cand_slot;
  KM_LAUNCH(c, launch_stream(dtype, kModeSwap, cfg, grid_for(c, cfg), sa, c.s));
  PointArgs pa = point_args(c);
  pa.cand_delta = cand_delta;
  pa.cand_slot = cand_slot;
  KM_LAUNCH(c, launch_fill_medoid_rows(pa, c.s));
  KmState h;
  r = read_state(c, &h);
  if (r != KM_OK) return r;
  if (best_delta) *best_delta = (h.best_cand < 0) ? __builtin_inf()
                                                  : (dtype != KM_F32 ? (double)h.best_i : h.best_d);
  if (best_slot) *best_slot = h.best_slot;
  if (best_cand) *best_cand = h.best_cand;
  return KM_OK;
}

km_status kmedoids_cache(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                         const int32_t* medoids, int32_t* near, int32_t* sec, void* dn, void* ds,
                         double* removal, void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  Ctx c;
  km_status r = check_common(D, dtype, n, n, ld, k, ws, ws_bytes, nullptr, &c);
  if (r != KM_OK) return r;
  if (!medoids) return fail(KM_E_INVALID, "medoids is NULL");
  c.s = static_cast<cudaStream_t>(stream);
  r = reset_state(c);
  if (r != KM_OK) return r;
  KM_CUDA(cudaMemcpyAsync(c.at<int32_t>(c.L.med), medoids, 4 * (size_t)k, cudaMemcpyDeviceToDevice, c.s));
  r = swap_setup(c);
  if (r != KM_OK) return r;
  if (near) KM_CUDA(cudaMemcpyAsync(near, c.at<int32_t>(c.L.near), 4 * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  if (sec) KM_CUDA(cudaMemcpyAsync(sec, c.at<int32_t>(c.L.sec), 4 * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  if (dn) KM_CUDA(cudaMemcpyAsync(dn, c.at<void>(c.L.dn), 4 * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  if (ds) KM_CUDA(cudaMemcpyAsync(ds, c.at<void>(c.L.ds), 4 * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  if (removal) {
    PointArgs pa = point_args(c);
    pa.out_double = removal;
    KM_LAUNCH(c, launch_removal_to_double(dtype, pa, c.s));
  }
  KmState h;
  return read_state(c, &h);
}

// Shared set-up of the two initialisations: argument checks, fixed-point
// scale of the matrix, kernel arguments over the workspace.
static km_status init_setup(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                            int32_t* medoids_out, void* ws, size_t ws_bytes, void* stream, Ctx* c,
                            InitArgs* ia) {
  g_err.clear();
  km_status r = check_common(D, dtype, n, n, ld, k, ws, ws_bytes, nullptr, c);
  if (r != KM_OK) return r;
  if (!medoids_out) return fail(KM_E_INVALID, "medoids_out is NULL");
  c->s = static_cast<cudaStream_t>(stream);
  r = reset_state(*c);
  if (r != KM_OK) return r;
  if (dtype == KM_F32) {
    r = scan_matrix(*c);
    if (r != KM_OK) return r;
  }
  memset(ia, 0, sizeof(*ia));
  ia->D = D;
  ia->ld = ld;
  ia->n = (int)n;
  ia->k = k;
  ia->fshift = c->fshift;
  ia->med = c->at<int32_t>(c->L.med);
  ia->dn = c->at<void>(c->L.bdn);
  ia->flags = c->at<uint8_t>(c->L.is_med);
  ia->csum = c->at<long long>(c->L.cand_gain);  // n_pad doubles >= n/32 sums
  ia->gains = c->at<double>(c->L.gains);
  ia->st = c->st();
  return KM_OK;
}

static km_status init_finish(Ctx& c, int32_t* medoids_out) {
  KmState h;
  KM_CUDA(cudaMemcpyAsync(&h, c.st(), sizeof(KmState), cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  if (h.error) return fail(KM_E_INVALID, "an initialisation step had an empty subsample");
  KM_CUDA(cudaMemcpyAsync(medoids_out, c.at<int32_t>(c.L.med), 4 * (size_t)c.k,
                          cudaMemcpyDeviceToDevice, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  return KM_OK;
}

km_status kmedoids_init_weighted(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                                 const double* u, int32_t* medoids_out, void* ws,
                                 size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_init_weighted");
  Ctx c;
  InitArgs ia;
  if (!u) return fail(KM_E_INVALID, "u is NULL");
  km_status r = init_setup(D, dtype, n, ld, k, medoids_out, ws, ws_bytes, stream, &c, &ia);
  if (r != KM_OK) return r;
  std::vector<double> hu((size_t)k);
  KM_CUDA(cudaMemcpyAsync(hu.data(), u, 8 * (size_t)k, cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  for (int t = 0; t < k; ++t)
    if (!(hu[t] >= 0.0 && hu[t] < 1.0))
      return fail(KM_E_INVALID, "u[%d] = %g is not in [0, 1)", t, hu[t]);
  ia.u = u;
  KM_LAUNCH(c, launch_init_weighted(dtype, ia, c.s));
  return init_finish(c, medoids_out);
}

km_status kmedoids_init_lab(const void* D, int32_t dtype, int64_t n, int64_t ld, int32_t k,
                            int32_t s, const int32_t* ranks, int32_t* medoids_out,
                            double* gains_host, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nv("kmedoids_init_lab");
  Ctx c;
  InitArgs ia;
  if (!ranks) return fail(KM_E_INVALID, "ranks is NULL");
  if (s < 1) return fail(KM_E_INVALID, "s must be >= 1 (got %d)", s);
  if (s > 4096 || k > 8192)
    return fail(KM_E_UNSUPPORTED, "LAB supports s <= 4096 and k <= 8192 (s=%d, k=%d)", s, k);
  km_status r = init_setup(D, dtype, n, ld, k, medoids_out, ws, ws_bytes, stream, &c, &ia);
  if (r != KM_OK) return r;
  // every step: ranks in [0, n - t) or negative (unused), distinct, >= 1 used
  std::vector<int32_t> hr((size_t)k * s);
  KM_CUDA(cudaMemcpyAsync(hr.data(), ranks, 4 * hr.size(), cudaMemcpyDeviceToHost, c.s));
  KM_CUDA(cudaStreamSynchronize(c.s));
  std::vector<int32_t> stamp((size_t)n, -1);
  for (int t = 0; t < k; ++t) {
    int used = 0;
    for (int j = 0; j < s; ++j) {
      const int32_t v = hr[(size_t)t * s + j];
      if (v < 0) continue;
      if ((int64_t)v >= n - t)
        return fail(KM_E_INVALID, "LAB rank %d of step %d is outside [0, %lld)", v, t,
                    (long long)(n - t));
      if (stamp[v] == t) return fail(KM_E_INVALID, "LAB rank %d repeated in step %d", v, t);
      stamp[v] = t;
      ++used;
    }
    if (!used) return fail(KM_E_INVALID, "LAB step %d has an empty subsample", t);
  }
  ia.s = s;
  ia.ranks = ranks;
  KM_LAUNCH(c, launch_init_lab(dtype, ia, c.s));
  r = init_finish(c, medoids_out);
  if (r != KM_OK) return r;
  if (gains_host) {
    KM_CUDA(cudaMemcpyAsync(gains_host, c.at<double>(c.L.gains), 8 * (size_t)k,
                            cudaMemcpyDeviceToHost, c.s));
    KM_CUDA(cudaStreamSynchronize(c.s));
  }
  return KM_OK;
}

}  // extern "C"

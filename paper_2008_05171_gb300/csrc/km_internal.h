// km_internal.h -- host-side interface between the C-ABI layer (km_api.cu)
// and the kernel translation units.  Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace km {

// NVTX range for the duration of a scope (phases of a call show up in
// profilers that record NVTX; without one attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct KmState;


// Streaming-kernel modes.
enum StreamMode { kModeSwap = 0, kModeBuild = 1 };

// SWAP pass flavours (what the last CTA decides after the pass).
enum SwapFlavour {
  kFastPAM1 = 0,  // best swap; accept iff Delta < -tol, else done
  kFastPAM2 = 1,  // as FastPAM1 + per-slot best swaps queued for later
  kFasterPAM = 2, // window of the cyclic scan; first improving candidate
  kEvalOnly = 3,  // evaluation only: best key written, no decision
  kCLARANS = 4    // window of the caller's draws; first improving draw,
                  // stop after maxneighbor consecutive failed draws
};

struct StreamArgs {
  const void* D;
  long long ld;
  int n;                // points (matrix columns)
  int m;                // candidate rows: n, or the locations of the bichromatic form
  int k;
  int k_pad;
  int n_pad;
  const uint8_t* is_med;
  // SWAP per-point cache (n_pad entries, padding holds sentinels)
  const void* dn;
  const void* ds;
  const int32_t* near;
  // BUILD nearest distance (n_pad entries)
  const void* bdn;
  int build_first;
  // removal loss [2][k_pad] and exact TD [2] (accumulator type)
  void* removal;
  void* td2;
  KmState* st;
  void* partials;       // Key[kMaxGrid]
  void* slot_partials;  // Key[kMaxGrid][k]   (FastPAM2)
  void* slot_best;      // Key[k]             (FastPAM2)
  int32_t* fp2_order;   // [k]                (FastPAM2)
  double* cand_delta;   // per-candidate outputs (index = output index)
  int32_t* cand_slot;
  double* cand_gain;    // BUILD per-candidate gains
  int flavour;          // SwapFlavour
  int win_rows;         // FasterPAM / FastCLARANS: positions per CTA
  const int32_t* draws; // FastCLARANS: candidate draws (DEVICE)
  long long draws_len;
  long long maxneighbor;
  int fshift;           // fixed-point exponent f of the SWAP sums (float data)
  double tol;
};

struct PointArgs {
  const void* D;
  long long ld;
  int n;          // points (matrix columns)
  int m;          // candidate rows: n, or the locations of the bichromatic form
  int k;
  int k_pad;
  int n_pad;
  int32_t* med;
  uint8_t* is_med;
  int32_t* near;
  int32_t* sec;
  void* dn;
  void* ds;
  void* bdn;
  void* removal;  // [2][k_pad]
  void* td2;      // [2]
  KmState* st;
  void* trace;    // TraceRec[trace_cap]
  int trace_cap;
  int build_first;
  int fp2_index;  // FastPAM2 extra-swap index
  double fp2_tol;
  const void* slot_best;      // Key[k] (FastPAM2)
  const int32_t* fp2_order;   // [k]    (FastPAM2)
  double* gains;              // BUILD gains per step [k]
  const double* cand_in;      // per-candidate values (k = 1 path)
  double* cand_delta;         // fill kernel outputs
  int32_t* cand_slot;
  double* out_double;         // accumulator -> double conversion target
  void* partials; // Key[kMaxGrid] scratch for grid reductions
  int fshift;     // fixed-point exponent f of the removal loss (float data)
  unsigned* scan; // matrix scan result: [0] max |d| bits, [1] invalid flag
};

// The eager variants (FasterPAM, FastCLARANS) as one persistent cooperative
// launch (km_eager.cu).
struct EagerArgs {
  const void* D;
  long long ld;
  int n;
  int k;
  int k_pad;
  int fshift;
  int32_t* med;
  uint8_t* is_med;
  int32_t* near;
  int32_t* sec;
  void* dn;
  void* ds;
  void* removal;          // [2][k_pad] fixed point / int64
  void* td2;              // [2] exact TD
  KmState* st;
  double* win_delta;      // [2][win_cap] per-position Delta of a window
  int32_t* win_slot;      // [2][win_cap] its best slot (-1: not evaluated)
  long long win_cap;
  int win_rows;           // largest window = grid x win_rows positions
  unsigned* bar;          // grid barrier: monotonic arrival count
  void* trace;            // TraceRec[trace_cap]
  int trace_cap;
  int flavour;            // kFasterPAM or kCLARANS
  const int32_t* draws;   // FastCLARANS draws (DEVICE)
  long long draws_len;
  long long maxneighbor;
  long long max_pos;      // FasterPAM: scan positions allowed (max_iter n)
  double tol;
};

size_t eager_smem(int k);
int eager_grid(int dtype, int k);  // co-resident CTAs, 0 if it cannot run
cudaError_t launch_eager(int dtype, int grid, const EagerArgs& a, cudaStream_t s);

// Incremental BUILD (km_build.cu): update passes and the commit of a step.
enum BuildMode {
  kBuildColsum = 0,  // step 0: distance sums over all rows
  kBuildFirst = 1,   // gains after step 0: all rows, d_n from the first medoid
  kBuildStep = 2     // later steps: the rows whose d_n dropped
};

struct BuildAux {
  unsigned cnt[2];               // listed points, by step parity (the update
                                 // after the commit of step t reads cnt[t & 1]
                                 // and clears cnt[(t & 1) ^ 1] for the next)
  unsigned gticket;              // column tiles done (last-block ticket)
  unsigned pad;
  unsigned long long rows_total; // rows the update passes streamed
};

struct BuildArgs {
  const void* D;
  long long ld;
  int n;
  int n_pad;
  int k;               // medoids to choose (length of med and gains)
  int fshift;          // fixed-point exponent f (float data)
  int first;           // commit of step 0
  int cur;             // parity of the step whose list is written / read
  KmState* st;
  BuildAux* aux;
  unsigned* tticket;   // [tiles] CTAs of each column tile done
  void* partials;      // Key[tiles] best non-medoid of each tile
  long long* cgain;    // [n_pad] fixed-point gain of every candidate
  int32_t* list;       // [n] points whose d_n dropped at the last commit
  uint32_t* lvn;       // [n] their new d_n (stored bits)
  uint32_t* lvo;       // [n] their old d_n (stored bits)
  void* bdn;           // [n_pad] d_n of every point
  int32_t* med;        // chosen medoids
  uint8_t* is_med;
  double* gains;       // BUILD gains per step [k] (may be NULL)
};

int build_update_groups(int n, int sms);
cudaError_t launch_build_update(int dtype, int mode, int groups, const BuildArgs& a,
                                cudaStream_t s);
cudaError_t launch_build_add(int dtype, const BuildArgs& a, cudaStream_t s);

// Initialisation kernels (Sec. 3.3): distance-weighted seeding and LAB.
struct InitArgs {
  const void* D;
  long long ld;
  int n;
  int k;
  int s;                 // LAB: subsample entries per step
  int fshift;            // fixed-point exponent f (float data)
  const double* u;       // weighted: k uniform numbers (DEVICE)
  const int32_t* ranks;  // LAB: k x s subsample ranks (DEVICE)
  int32_t* med;          // k chosen medoids (DEVICE)
  double* gains;         // LAB: each step's least gain (may be NULL)
  void* dn;              // n_pad distances to the nearest chosen medoid
  uint8_t* flags;        // n_pad drawn flags
  long long* csum;       // weighted: ceil(n/32) chunk weight sums
  KmState* st;
};

size_t init_lab_smem(int k, int s);
cudaError_t launch_init_weighted(int dtype, const InitArgs& a, cudaStream_t s);
cudaError_t launch_init_lab(int dtype, const InitArgs& a, cudaStream_t s);

// Launch configuration chosen for a (mode, k) pair.
struct StreamConfig {
  int rows;       // candidate rows per tile (R)
  int stages;     // ring depth (S)
  int minb;       // CTAs per SM the kernel is built for
  size_t smem;    // dynamic shared memory bytes
  int geometry;   // index into the geometry table (1-based)
};

// Returns false if no configuration fits (k too large).  tune > 0 forces a
// geometry of the table; forced_rows > 0 restricts the automatic choice.
// esize: bytes per stored matrix element (4, or 2 for the 16-bit form).
bool stream_config(int mode, int k, int flavour, int forced_rows, int tune, StreamConfig* cfg,
                   int esize = 4);

cudaError_t launch_stream(int dtype, int mode, const StreamConfig& cfg, int grid,
                          const StreamArgs& a, cudaStream_t s);

cudaError_t launch_cache_init(int dtype, const PointArgs& a, cudaStream_t s);
cudaError_t launch_apply(int dtype, const PointArgs& a, cudaStream_t s);
cudaError_t launch_build_commit(int dtype, const PointArgs& a, cudaStream_t s);
cudaError_t launch_fp2_try(int dtype, const PointArgs& a, cudaStream_t s);
cudaError_t launch_mark_medoids(const PointArgs& a, cudaStream_t s);
cudaError_t launch_reset_state(KmState* st, unsigned long long wait_ns, cudaStream_t s);
cudaError_t launch_build_handoff(KmState* st, KmState* saved, int32_t* med, int k,
                                 cudaStream_t s);
cudaError_t launch_swap_loop_cond(KmState* st, unsigned long long handle, int max_iter,
                                  cudaStream_t s);
cudaError_t launch_fill_medoid_rows(const PointArgs& a, cudaStream_t s);
cudaError_t launch_removal_to_double(int dtype, const PointArgs& a, cudaStream_t s);
cudaError_t launch_matrix_scan(const PointArgs& a, cudaStream_t s);
// Checks D (zero diagonal, bitwise symmetry, finite entries >= 0 for float
// data) and ORs the findings into *flags (1, 2, 4).
cudaError_t launch_matrix_check(int dtype, const void* D, long long ld, int n, unsigned* flags,
                                cudaStream_t s);

int device_sm_count();

cudaError_t launch_prearrange(const void* X, long long ldx, int n, int d, int n_pad, void* Xp,
                              cudaStream_t s);
cudaError_t launch_row_norms(const void* X, long long ldx, int n, int d, int n_pad, float* norms,
                             cudaStream_t s);

// Replace the thread-local message returned by kmedoids_last_error().
void set_last_error(const char* msg);

}  // namespace km

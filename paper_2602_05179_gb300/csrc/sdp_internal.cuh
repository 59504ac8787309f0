// sdp_internal.cuh -- internal declarations shared by the libsdp translation
// units (kernels + C-ABI layer).  Not part of the public ABI (include/sdp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdp.h"

namespace sdp {

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------- Split prep
// Per tour position i = 1..n one 16-byte record, read by every scenario of
// the tour (a warp-uniform broadcast load per DP step):
//   col = s_i - 1            (column of customer s_i in a demand row)
//   a   = c(0,s_i) - c(s_{i-1},s_i)   (0 for the second term when i = 1)
//   ce  = c(s_i, 0)
// With D(k) = sum_{m=1}^{k-1} c(s_m,s_{m+1}) and K(i) = J(i) - D(i), the
// recursion of Eq. eqdpA becomes
//   psi(p) = K(p) + a_{p+1},  K(i) = min_{p in window(i)} psi(p) + ce_i,
//   J(n)   = K(n) + D(n),
// so every FP32 operand stays at the scale of the depot legs rather than the
// whole tour length; D(n) is accumulated in FP64 once per tour.
struct __align__(16) StepRec {
  uint32_t col;
  float a;
  float ce;
  uint32_t pad;
};

struct TourPrep {
  StepRec* rec;     // [n]
  uint16_t* cols;   // [n] (col of each position, compact copy for copy-out)
  double* Dn;       // [1] tour length D(n) in FP64
};

// ----------------------------------------------------------------- kernels
// status bits are OR-ed into *status (a per-device __device__ word).

// one CTA per tour; coords or dist mode
void launch_tour_prep(const int32_t* tour, int n, const float* coords,
                      const float* dist, TourPrep prep, uint32_t* status,
                      uint32_t* reset_word, cudaStream_t st);

struct SplitPlainArgs {
  int n, Q;
  int64_t S;
  const StepRec* rec;
  const double* Dn;
  const int32_t* demands;
  float* cost;
  void* pred;           // nullable
  int pred_dtype;
  float* kscratch;      // [(n+1) * nslots], K(p) of the scenario in slot
  int32_t* pscratch;    // [n * nslots] preds when pred == NULL and hist != NULL
  int64_t nslots;
  unsigned long long* hist;  // [2n] or NULL (route start / end counts)
  const uint32_t* fb_list;   // NULL: all scenarios; else list of scenario ids
  const uint32_t* fb_count;  // [1] number of entries in fb_list
  uint32_t* status;
  int soft;                  // soft capacity: every p, beta per unit above Q
  float beta;
};
void launch_split_plain(const SplitPlainArgs& a, int grid, cudaStream_t st);
int plain_grid(int device_sms);

struct SplitDequeArgs {
  int n, Q;
  int64_t S;
  const StepRec* rec;
  const uint16_t* cols;
  const double* Dn;
  const int32_t* demands;
  float* cost;          // nullable in the fused backward
  void* pred;           // nullable
  int pred_dtype;
  unsigned long long* hist;  // [2n] or NULL: fused backtrack histograms
  uint32_t* fb_list;    // [S] scenario ids that need the per-scenario path
  uint32_t* fb_count;   // [1]
  uint32_t* status;
  int soft;             // soft capacity: beta per unit of route load above Q
  float beta;
};
struct DequeConfig {
  int warps;        // warps per CTA
  int ring;         // deque ring entries per scenario (8, 16, 32)
  int qbytes;       // 1 (uint8 staging) or 2 (uint16 staging)
  int row_stride;   // bytes per staged demand row (shared-memory staging)
  bool rec_in_smem; // tour records copied to shared memory (n <= 4096)
  bool tmem;        // demand rows staged in tensor memory (one CTA per SM)
  size_t smem;      // dynamic shared memory per CTA
};
bool deque_supported(int n, int Q);
// pred_bytes: size of one output predecessor (0 when none are written);
// allow_tmem: stage demands in TMEM when a row fits 128 columns.
DequeConfig deque_config(int n, int Q, int warps, int ring, bool hist, int pred_bytes,
                         bool allow_tmem);
// returns 0 or a cudaError_t
int launch_split_deque(const SplitDequeArgs& a, const DequeConfig& c, int grid,
                       cudaStream_t st);
int deque_max_ctas_per_sm(const DequeConfig& c, bool hist, int pred_dtype,
                          bool want_pred, int* out);
// The default TMEM launch c made wide (17..24 warps, every one staging its
// tile in TMEM) when that many take every tile in one round where 16 would
// need two, and the rows fit; direct_ok: no predecessors, or predecessors stored 4 per lane
// (n % 4 == 0, 16-byte aligned rows).  Returns c itself otherwise.
DequeConfig deque_config_wide(const DequeConfig& c, int n, int Q, int64_t S, bool direct_ok,
                              int sms);
// Fused adjoint and forward with TMEM-staged rows: warps per CTA (16..24)
// for S scenarios on sms SMs (more than 16 only for a single round), 0 where
// rows do not fit 16 warps' columns; the [word][lane] delta
// scratch it needs; the launch (hist set, cost / pred unused).
int split_tmem_adj_warps(int n, int Q, int64_t S, int sms);
size_t split_tmem_adj_scratch_bytes(int n, int Q, int sms);
int launch_split_tmem_adj(const SplitDequeArgs& a, int warps, uint32_t* dscratch, int sms,
                          cudaStream_t st);

// batched Split (persistent work queue over (tour, 32-scenario tile) items)
struct BatchKernelArgs {
  int B, Q, n_max;
  int64_t S;
  const int32_t* n;          // [B]
  const int64_t* dem_off;    // [B] element offset of tour b's [S, n_b] block
  const int64_t* rec_off;    // [B] offset of tour b's StepRecs
  const int32_t* order;      // [B] tours by decreasing n
  const StepRec* rec;
  const double* Dn;          // [B]
  const int32_t* demands;
  float* costs;              // [B*S]
  unsigned long long* counter;
  unsigned long long* fb_list;  // [B*S] global scenario ids b*S+s
  uint32_t* fb_count;
  uint32_t* status;
};
// warps == 0: tensor-memory staging (warps per CTA chosen from n_max);
// ns: scenarios per lane of the shared-memory kernel (1 or 2)
size_t batch_smem(int n_max, int Q, int warps, int ring, int ns);
int batch_tmem_warps(int n_max, int Q);
struct BatchPrepArgs {
  const int32_t* n;
  const int64_t* tour_off;
  const int64_t* coord_off;
  const int64_t* rec_off;
  const int32_t* tours;
  const float* coords;
  StepRec* rec;
  double* Dn;
  unsigned long long* counter;  // reset to 0 by the prep kernel
  uint32_t* fb_count;           // reset to 0 by the prep kernel
  uint32_t* status;
};
void launch_batch_prep(const BatchPrepArgs& a, int B, cudaStream_t st);
void launch_batch_means(const float* costs, int B, int64_t S, double* means, cudaStream_t st);
void launch_batch_count(const BatchPrepArgs& a, int B, int64_t S, int Q, const int64_t* dem_off,
                        const int32_t* demands, unsigned long long* total, cudaStream_t st);
struct BatchFallbackArgs {
  int Q;
  int64_t S;
  const int32_t* n;
  const int64_t* dem_off;
  const int64_t* rec_off;
  const StepRec* rec;
  const double* Dn;
  const int32_t* demands;
  float* costs;
  const unsigned long long* fb_list;
  const uint32_t* fb_count;
  float* kscratch;   // [(n_max+1) * nslots]
  int64_t nslots;
};
void launch_batch_fallback(const BatchFallbackArgs& a, cudaStream_t st);

// Warp-per-scenario recomputation of flagged hard-capacity scenarios
// (split_rescue.cu), one tour or a batched plan's entries; the same FP32
// results as the plain kernel.
struct RescueArgs {
  int batched;
  int Q;
  int64_t S;
  int n_max;                   // longest tour (shared memory per warp: 8 (n_max+1) bytes)
  // one tour
  int n1;
  const uint32_t* fb_list1;    // [*fb_count] scenario ids
  float* cost;                 // [S]
  void* pred;                  // [S, n] or NULL
  int pred_dtype;
  // batched: entry g = b*S + s
  const int32_t* n;
  const int64_t* rec_off;
  const int64_t* dem_off;
  const unsigned long long* fb_list;
  float* costs;                // [B*S]
  // both
  const StepRec* rec;
  const double* Dn;            // [1] or [B]
  const int32_t* demands;
  const uint32_t* fb_count;
  uint32_t* status;
};
bool rescue_supported(int n_max);
// max_work: the most entries the list can hold (sizes the grid)
int launch_split_rescue(const RescueArgs& a, int64_t max_work, cudaStream_t st);
int launch_split_batch(const BatchKernelArgs& a, int warps, int ring, int ns, int grid,
                       cudaStream_t st, int* occ_out);

// Split with demands streamed in tour order (SDP_ALGO_STREAM): a pre-pass
// narrows and permutes the demand rows, then the DP streams them.
constexpr int kStreamMaxN = 2048;
struct StreamArgs {
  int n, Q;
  int64_t S;
  const StepRec* rec;       // [n]
  const uint16_t* cols;     // [n] column (customer - 1) of each tour position
  const double* Dn;
  const int32_t* demands;   // [S, n] by customer, 16-byte aligned
  unsigned char* qt;        // [S, stride] narrowed demands in tour order
  int64_t stride;           // bytes per qt row (stream_row_stride)
  uint32_t* tflags;         // [ceil(S/32)] rows with a demand above Q, per tile
  float* cost;
  void* pred;               // nullable
  int pred_dtype;
  uint32_t* fb_list;        // [S] scenarios recomputed by the plain kernel
  uint32_t* fb_count;
  uint32_t* status;
  int ctas_per_sm;          // CTAs per SM (0 = 1)
  uint64_t wait_ns;         // a DP warp's wait for a tile gives up after this
  int stall;                // fault injection (tests): producers publish no tile
};
bool stream_supported(int n, int Q);
// batched plan over tour-ordered row slots (one ring of slots per SM)
struct BatchStreamArgs {
  int B, Q;
  int64_t S;
  const int32_t* n;          // [B]
  const int64_t* dem_off;    // [B] element offsets, multiples of 4
  const int64_t* rec_off;    // [B]
  const int32_t* order;      // [B] tours by decreasing n
  const StepRec* rec;
  const double* Dn;          // [B]
  const int32_t* demands;    // 16-byte aligned
  float* costs;              // [B*S]
  unsigned long long* counter;  // group queue (reset by the prep kernel)
  unsigned long long* fb_list;
  uint32_t* fb_count;
  uint32_t* status;
  unsigned char* qt;         // batch_stream_qt_bytes
  int64_t stride_max;        // bytes per row slot
};
bool batch_stream_supported(int n_max, int Q);
int64_t batch_stream_stride(int n_max, int Q);
size_t batch_stream_qt_bytes(int n_max, int Q);
int launch_split_batch_stream(const BatchStreamArgs& a, cudaStream_t st);
// bytes per tour-ordered row: n narrowed demands (uint8 for Q <= 254, else
// uint16), >= 16 bytes of slack for the one-block look-ahead, 32-byte rows
__host__ __device__ inline int64_t stream_row_stride(int n, int Q) {
  const int64_t qb = Q <= 254 ? 1 : 2;
  return ((int64_t)n * qb + 16 + 31) / 32 * 32;
}
size_t stream_qt_bytes(int n, int Q, int64_t S);
int launch_split_stream(const StreamArgs& a, cudaStream_t st);

// Pipelined Split (SDP_ALGO_PIPE, and the batched plans' pipelined kernel):
// producer warps narrow and permute demand rows into a per-SM ring of
// tour-ordered tile slots kept small enough to stay in L2, DP warps run the
// recursion on them.  One tour (batched = 0: n1, cols, rec, Dn[0]; cost and
// pred by scenario) or a batched plan (batched = 1: n, dem_off, rec_off,
// order by tour; costs [B*S]; no predecessors).
constexpr int kPipeMaxN = 1024;
struct PipeArgs {
  int batched;
  int B, Q;
  int64_t S;
  int n1;                      // one tour: n
  const uint16_t* cols;        // one tour: [n] column (customer - 1) of each position
  const int32_t* n;            // batched: [B]
  const int64_t* dem_off;      // batched: [B] element offsets, multiples of 4
  const int64_t* rec_off;      // batched: [B]
  const int32_t* order;        // batched: [B] tours by decreasing n
  const StepRec* rec;
  const double* Dn;            // [B]
  const int32_t* demands;      // 16-byte aligned
  float* cost;                 // [B*S]
  void* pred;                  // one tour only: [S*n] or NULL
  int pred_dtype;
  unsigned char* qt;           // slot ring, pipe_ring_bytes
  int nslot;                   // slots per CTA (set by launch_split_pipe)
  int n_max;                   // batched: the longest tour
  int soft;                    // one tour: soft capacity, beta per unit of route load above Q
  float beta;
  int64_t stride;              // bytes per slot row (pipe_row_stride of the longest tour)
  unsigned long long* counter; // group queue, zero at launch
  uint32_t* fb_count;
  uint32_t* fb_list1;          // one tour: [S] scenario ids for the plain kernel
  unsigned long long* fb_list; // batched: [B*S] global ids b*S+s
  uint32_t* status;
  uint64_t wait_ns;            // a bounded wait gives up after this
  int stall;                   // fault injection (tests): producers publish no tile
};
bool pipe_supported(int n, int Q);
// bytes per tour-ordered slot row: n narrowed demands (uint8 for Q <= 254,
// else uint16) rounded up to 32 bytes
__host__ __device__ inline int64_t pipe_row_stride(int n, int Q) {
  const int64_t qb = Q <= 254 ? 1 : 2;
  return ((int64_t)n * qb + 31) / 32 * 32;
}
// CTAs of a launch (one per SM at most, none without work) and the slot
// ring they need
int pipe_grid(int64_t S, int B, bool batched);
size_t pipe_ring_bytes(int n_max, int Q, int64_t S, int B, bool batched);
int launch_split_pipe(const PipeArgs& a, cudaStream_t st);

// Fleet-limited Split (at most K routes, K <= 64): one warp per scenario
// with the route-count layers across lanes, and a one-thread-per-scenario
// layered kernel (PLAIN, and the recomputation of flagged scenarios).
constexpr int kFleetMaxK = 64;
struct SplitFleetArgs {
  int n, Q, K;
  int64_t S;
  const StepRec* rec;
  const double* Dn;
  const int32_t* demands;
  float* cost;               // [S]
  int32_t* nroutes;          // [S] or NULL
  uint8_t* route;            // [S*n] or NULL: route of each position, 0xFF if infeasible
  uint16_t* dscratch;        // warp kernel with routes: fleet_dscratch_elems
  uint32_t* fb_list;         // warp kernel: flagged scenarios; plain: NULL = all S
  uint32_t* fb_count;
  float* kscratch;           // plain: [nslots * 2 * (n+1)]
  uint16_t* pscratch;        // plain with routes: [nslots * K * n]
  int64_t nslots;
  uint32_t* status;
};
struct FleetConfig {
  int warps;  // warps per CTA (0: the tour's records do not fit)
  int grid;
};
FleetConfig fleet_config(int n, int K, int64_t S);
size_t fleet_dscratch_elems(int n, int K, const FleetConfig& c);
int launch_split_fleet(const SplitFleetArgs& a, const FleetConfig& c, cudaStream_t st);
int launch_split_fleet_plain(const SplitFleetArgs& a, cudaStream_t st);
// the flagged scenarios (fb_list), one warp each; the plain kernel's bits
bool fleet_rescue_supported(int n);
int launch_split_fleet_rescue(const SplitFleetArgs& a, cudaStream_t st);

// arc counting (capacity-feasible (p,i) pairs)
void launch_count_arcs(int n, int Q, int64_t S, const StepRec* rec,
                       const int32_t* demands, int64_t* arcs,
                       unsigned long long* total, int grid, cudaStream_t st);

// FP64 mean of a float array, deterministic (fixed blocking and order)
constexpr int kMeanBlocks = 512;
void launch_mean(const float* x, int64_t count, double* partial /*[kMeanBlocks]*/,
                 double* out, cudaStream_t st);

// adjoint assembly: grad[(n+1)^2] = counts / S * (*grad_mean)
void launch_grad_assemble(int n, int64_t S, const int32_t* tour,
                          const unsigned long long* hist, const float* grad_mean,
                          float* grad, int64_t* hist_out, cudaStream_t st);
void launch_backtrack_hist(int n, int64_t S, const void* pred, int pred_dtype,
                           unsigned long long* hist, uint32_t* status,
                           cudaStream_t st);

// reinsertion
struct ReinsertArgs {
  int algo;  // SDP_REINSERT_*
  int T, U, I0;
  float h, p, c;
  int64_t S;
  const float* fixed;
  const float* table;
  const int32_t* cons;
  float* value;
  uint8_t* policy;
  float* value0;
  uint32_t* status;
  uint32_t* dscratch;  // lane kernel with a policy: reinsert_lane_scratch_bytes
  int n_routes;               // route options per day (0: the two-action DP)
  const float* route_cost;    // [T * n_routes]
  const int32_t* route_cap;   // [S * T * n_routes]
};
int launch_reinsert(const ReinsertArgs& a, cudaStream_t st);
// one-scenario-per-lane kernel: shapes it runs, its shared memory and the
// decision scratch it needs when the policy is wanted
bool reinsert_lane_supported(int T, int U, int n_routes);
size_t reinsert_lane_smem(int T, int U, bool table);
size_t reinsert_lane_smem_for(int T, int U, bool table, int warps, int n_routes);
int reinsert_lane_warps(int T, int U, bool table, int n_routes);
size_t reinsert_lane_scratch_bytes(int T, int U);

int num_sms();

// Host-side fault injection (sdp_set_fault_inject / SDP_FAULT_INJECT): true
// if the next plan / search allocation is to fail; the stall time of the next
// streaming launch (0: none); the pending failure of an operator call (0 or
// an SDP_ERR_* code, with the message set).
bool fault_alloc();
uint64_t fault_stall_ns();
int fault_call_hook();
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // device waits give up after 2 s

}  // namespace sdp

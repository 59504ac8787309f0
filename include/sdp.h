/*
 * sdp.h -- C ABI of libsdp: scenario-batched Bellman (min-plus) kernels for
 * GB300 (sm_103a), after arXiv 2602.05179, "From Sequential to Parallel:
 * Reformulating Dynamic Programming as GPU Kernels for Large-Scale Stochastic
 * Combinatorial Optimization".
 *
 * Operators
 *   Split (Sec. 2 "Instantiation A", Eq. eqdpA; Algorithms "GPU Splitting"
 *   and "2D Kernel for Splitting"): for a giant tour s_1..s_n, capacity Q and
 *   S demand scenarios, per scenario
 *       J(0) = 0,  J(i) = min_{p<i, load(s_{p+1..i}) <= Q} J(p) + W(p,i),
 *       W(p,i) = c(0,s_{p+1}) + sum_{k=p+1}^{i-1} c(s_k,s_{k+1}) + c(s_i,0),
 *   returning cost J(n), the predecessor array and the FP64 scenario mean.
 *   Reinsertion (Sec. 2 "Instantiation B", Eq. eqdp2; Algorithm
 *   "SolveBatchDP"): one customer, order-up-to level U, horizon T, per
 *   scenario the backward DP over inventory states 0..U with the two actions
 *   "no delivery" and "deliver up to U", returning the value from I0, the
 *   optimal policy and the FP64 scenario mean.
 *
 * Conventions (every entry point)
 *   - Array arguments are DEVICE pointers owned by the caller unless a field
 *     says "host".  The library never frees them and never keeps them after
 *     the call returns (plans keep the pointers given at creation).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Outputs are valid once the stream
 *     has reached the call.  Argument checks that need no device data happen
 *     before anything is launched; on error nothing is launched.
 *   - The return value is a status code (SDP_OK, SDP_WARN_*, SDP_ERR_*).
 *     sdp_last_error() gives a thread-local message for the last failure.
 *   - Conditions found by the kernels (a demand above Q, a negative demand or
 *     consumption) are raised in a per-device status word read with
 *     sdp_device_status() (which synchronises the device).
 *   - Eager calls never allocate device memory: scratch comes from the
 *     caller's `workspace` (size from the matching *_workspace_bytes query).
 *     Plans own device memory from sdp_split_plan_create until
 *     sdp_plan_destroy.
 *   - Calls on distinct streams are thread-safe; a plan must not be run
 *     concurrently with itself.
 */
#ifndef SDP_H_
#define SDP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDP_VERSION 1

/* status codes */
#define SDP_OK 0
#define SDP_WARN_INFEASIBLE 1     /* some scenario is infeasible (cost +inf) */
#define SDP_ERR_INVALID_ARG (-1)  /* bad size, null or host pointer, ... */
#define SDP_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define SDP_ERR_OOM (-3)          /* plan allocation failed */
#define SDP_ERR_WORKSPACE (-4)    /* workspace missing or too small */
#define SDP_ERR_UNSUPPORTED (-5)  /* valid but not supported (see field docs) */
#define SDP_ERR_DEVICE_CHECK (-6) /* a kernel's own bounds check fired */

/* device status word bits (sdp_device_status) */
#define SDP_FLAG_INFEASIBLE 1u     /* a Split scenario had a demand > Q */
#define SDP_FLAG_NEG_INPUT 2u      /* a negative demand / consumption was read */
#define SDP_FLAG_DEVICE_CHECK 4u   /* an internal bounds check fired */
#define SDP_FLAG_FALLBACK 8u       /* a scenario took the per-scenario path */

/* Split algorithms */
#define SDP_ALGO_AUTO 0   /* PIPE where it applies (hard or soft capacity,
                             n <= 1024,
                             Q <= 32767, 16-byte aligned device demands or
                             host demands, warps_per_cta = 0, ring 0 or 16);
                             else DEQUE when a demand row fits 512 bytes
                             (uint8 for Q <= 254, else uint16), STREAM for
                             longer rows it supports, else DEQUE; PLAIN when
                             none applies */
#define SDP_ALGO_PLAIN 1  /* one thread per scenario, demands read straight
                             from HBM, every feasible arc (p,i) relaxed in
                             turn: the min-plus column product of Eq. eqdpA */
#define SDP_ALGO_DEQUE 2  /* warp tile of 32 scenarios staged in shared
                             memory; the window minimum is kept in a monotone
                             deque (the linear split of Algorithm "2D Kernel
                             for Splitting"); needs Q <= 32767 */
#define SDP_ALGO_STREAM 3 /* the DEQUE recursion with the gather by customer
                             done once up front: a pre-pass narrows the
                             demands (uint8 for Q <= 254, else uint16) into
                             tour order in the workspace, then one lane per
                             scenario streams its row from HBM; needs
                             n <= 2048, Q <= 32767 and 16-byte aligned
                             demands.  The workspace grows by about
                             S * (n + 48) bytes (x2 for uint16) */

#define SDP_ALGO_PIPE 4   /* the DEQUE recursion fed by producer warps of the
                             same CTA, which narrow and permute each tile's
                             demand rows into tour order in a small ring of
                             tile slots that stays in L2 (no pre-pass over
                             HBM), with 23 DP warps per SM; predecessors
                             leave through a shared-memory transpose as row
                             segments.  Hard or soft capacity; needs
                             1 <= n <= 1024, Q <= 32767 and 16-byte aligned
                             demands; the
                             workspace grows by at most
                             SMs * 32 * 32 * ceil32(n * qb) bytes (qb = 1 for
                             Q <= 254, else 2): 78 MB at n = 500 on 152 SMs,
                             less when a CTA's share of the tiles is below
                             16 (two slots per tile of its share, 2 to 32) */

/* predecessor dtypes */
#define SDP_PRED_U16 1    /* uint16, requires n < 65535 */
#define SDP_PRED_I32 2    /* int32 */

int sdp_version(void);
const char* sdp_last_error(void);

/* Measurement hook.  start/stop are cudaEvent_t handles (as void*) created
 * by the caller; the calling thread's NEXT operator call records `start` on
 * its stream just before launching its dominant kernel (the DP kernel) and
 * `stop` just after it, then forgets them.  NULL, NULL disables.  Errors:
 * SDP_ERR_INVALID_ARG if exactly one is NULL. */
int sdp_set_profile_events(void* start, void* stop);

/* Launch shape of the DP kernel of the calling thread's last sdp_split_eval
 * or sdp_split_backward call: warps per CTA and CTAs (0, 0 for the STREAM
 * path, whose CTAs mix producer and DP warps; 0, 0 before any call).  The
 * shape is chosen from n, Q, S and the SM count, so a test can check that
 * the launch it means to exercise is the one that ran.  Host-side only;
 * always SDP_OK. */
int sdp_last_launch(int32_t* warps_per_cta_out, int32_t* ctas_out);

/* Reads (and with clear != 0 resets) the status word of the current device.
 * Synchronises the device.  *flags_out receives SDP_FLAG_* bits. */
int sdp_device_status(int clear, uint32_t* flags_out);

/* ------------------------------------------------------------------ Split */
/* One giant tour, S scenarios.
 * Exactly one of coords / dist is non-NULL:
 *   coords [(n+1)*2] fp32, (x,y) per node, node 0 = depot: c(a,b) is the fp32
 *          Euclidean distance (IEEE sqrt, no contraction);
 *   dist   [(n+1)*(n+1)] fp32 row-major, c(a,b) = dist[a*(n+1)+b].
 * The destination depot n+1 is the same node as the depot 0.
 * demands [S*n] int32, demands[s*n + c-1] = demand of customer c in scenario
 *   s (indexed by customer id; the tour permutes them).  Device memory, or
 *   page-locked host memory the device can address (cudaHostAlloc, or
 *   cudaHostRegister with cudaHostRegisterMapped), which must stay unchanged
 *   until the call's work on the stream has finished.  With host demands,
 *   sdp_split_eval copies them in chunks of 65,536 scenarios into two staging
 *   buffers (part of its workspace, which is then larger) on a copy stream
 *   of the library's own, each chunk's copy overlapping the evaluation of the
 *   previous one; the copy stream and its events are created on the first
 *   such call on a device and kept until the process exits, and such calls
 *   are enqueued one at a time.  sdp_split_count_arcs and
 *   sdp_split_backward read host demands in place over the host link.
 *   A demand above Q
 *   makes the scenario infeasible: cost +inf, predecessors -1 (0xFFFF for
 *   uint16), SDP_FLAG_INFEASIBLE raised.  Negative demands raise
 *   SDP_FLAG_NEG_INPUT and are read as 0.
 * Route costs are FP32 (computed as the DP of K(i) = J(i) - D(i), D the
 *   prefix tour length, which keeps every FP32 operand small); the tour
 *   length D(n) is accumulated in FP64; the mean is FP64.
 */
typedef struct sdp_split_args {
  int32_t n;              /* customers, n >= 0 (DEQUE: n <= 65534) */
  int32_t Q;              /* capacity, Q > 0 */
  int64_t S;              /* scenarios, S >= 0 */
  const int32_t* tour;    /* [n], permutation of 1..n (not checked) */
  const float* coords;    /* [(n+1)*2] or NULL */
  const float* dist;      /* [(n+1)*(n+1)] or NULL */
  const int32_t* demands; /* [S*n] */
  float* cost_out;        /* [S], required: J_s(n) */
  void* pred_out;         /* [S*n] or NULL: pred[s*n+i-1] = argmin p of J(i),
                             the smallest p on exact ties */
  int32_t pred_dtype;     /* SDP_PRED_U16 or SDP_PRED_I32 (ignored if no preds) */
  int32_t algo;           /* SDP_ALGO_* */
  double* mean_out;       /* [1] or NULL: (1/S) sum_s cost[s], +inf if any
                             scenario is infeasible */
  void* workspace;        /* device scratch, >= sdp_split_workspace_bytes */
  size_t workspace_bytes;
  int32_t warps_per_cta;  /* DEQUE tuning: 0 = default (demand rows staged in
                             tensor memory when a row fits 512 bytes, 16
                             warps per SM; else shared memory, up to 4 warps
                             per CTA as the rows fit); 1..8 = shared-memory
                             staging with that many warps per CTA (AUTO then
                             stays on DEQUE).  Ignored by STREAM */
  int32_t ring;           /* DEQUE tuning: deque ring entries per scenario,
                             0 = default, else 8, 16 or 32 */
  int32_t capacity_mode;  /* SDP_CAPACITY_HARD (0, Eq. eqdpA) or
                             SDP_CAPACITY_SOFT */
  float overload_penalty; /* SOFT: cost per unit of route load above Q
                             (finite, >= 0) */
} sdp_split_args;

/* Capacity modes.  SOFT is the penalised load of the paper's CVRPSD model:
 * every split is allowed and a route whose load exceeds Q pays
 * overload_penalty per unit of excess,
 *     J(i) = min_{0<=p<i} J(p) + W(p,i) + beta * max(0, load(s_{p+1..i}) - Q).
 * No scenario is infeasible.  PLAIN relaxes all n(n+1)/2 pairs (p,i); DEQUE
 * (tensor-memory staging, rows of at most 512 bytes) keeps the hard window in
 * its deque and the entries that left it as one running minimum of
 * psi(p) - beta L(p) (with equal slopes, an expired entry's penalised cost
 * is that value plus beta (L(i) - Q)), O(1) per position; PIPE runs the same
 * recursion with the same FP32 operations (the DEQUE soft kernel's bits) and
 * sends a scenario whose prefix load reaches 2^16, or that holds a demand
 * above 255 (Q <= 254) or 32767, to PLAIN.  AUTO takes PIPE where it applies,
 * else DEQUE, else PLAIN; STREAM, plans and the adjoint take HARD only
 * (SDP_ERR_UNSUPPORTED). */
#define SDP_CAPACITY_HARD 0
#define SDP_CAPACITY_SOFT 1

size_t sdp_split_args_size(void);
size_t sdp_split_workspace_bytes(const sdp_split_args* a);
int sdp_split_eval(const sdp_split_args* a, void* stream);

/* Split evaluation that allocates nothing, for callers that cannot hand the
 * library device memory beyond their inputs and outputs: host programs that
 * own every device allocation and pass a solver only the buffers it reads and
 * writes (plugins, embedded solvers), or latency-critical loops where a
 * cudaMalloc / cudaFree would synchronize the device.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Same arguments, results and errors as sdp_split_eval, except that
 * a->workspace / a->workspace_bytes are ignored: the scratch is a fixed
 * device array of SDP_NOALLOC_SCRATCH_BYTES inside the library, which every
 * device that loads the library holds until the process exits.
 *   - Calls whose workspace (sdp_split_workspace_bytes) exceeds that size are
 *     rejected with SDP_ERR_UNSUPPORTED and nothing is launched (at n = 500,
 *     algo DEQUE, about 2 million scenarios fit; algo PLAIN needs more).
 *     The scratch holds the workspace of sdp_split_workspace_bytes, whose
 *     large terms are: the plain kernel's fallback rows, (n+1) * min(S,4096)
 *     * 4 bytes (above 16 MiB from n = 1023 on, so DEQUE calls with
 *     S >= 4096 and long rows are rejected there); 4 * S bytes of fallback
 *     list; STREAM's tour-ordered rows, S * (n + 48) bytes or so (AUTO takes
 *     STREAM for n > 512); and with demands in page-locked host memory two
 *     staging buffers of min(S, 65536) * n * 4 bytes each (rejected from
 *     n = 32 on at S >= 65536).  Give such calls a workspace through
 *     sdp_split_eval instead.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it for
 *     the life of the process; make that first call before any stream
 *     capture.  The cached address belongs to the device's primary context:
 *     after cudaDeviceReset on that device the next call would pass a stale
 *     address, so do not use this entry point across a device reset (the
 *     status word that every entry point uses is cached the same way).
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call resets what must start at zero (the fallback counter).  Calls
 *     that overlap on the GPU (other streams, other host threads) race on it:
 *     serialise them. */
#define SDP_NOALLOC_SCRATCH_BYTES (16u << 20)
int sdp_split_eval_noalloc(const sdp_split_args* a, void* stream);

/* Fleet-limited Split: at most max_routes routes per scenario (Appendix A,
 * extensive model, constraint eq:fleet_size -- the giant-tour example there
 * has "three vehicles available"), hard capacity as in Eq. eqdpA.  With
 * J_k(i) the cost of serving positions 1..i with exactly k routes,
 *     J_k(i) = min over capacity-feasible p < i of J_{k-1}(p) + W(p,i),
 *     J_0(0) = 0, J_0(i > 0) = J_k(0) = +inf,  cost = min_{k <= K} J_k(n),
 * ties to the smallest p at every (k, i), then to the fewest routes.
 *   a:           as for sdp_split_eval, with pred_out = NULL, hard capacity,
 *                device demands, algo SDP_ALGO_AUTO (one warp per scenario,
 *                the route counts across its lanes) or SDP_ALGO_PLAIN (one
 *                thread per scenario, every feasible p of every layer; the
 *                same FP32 operations and bits); cost_out [S] fp32 (+inf
 *                where no split into at most max_routes routes fits Q, or a
 *                demand exceeds Q: SDP_WARN_INFEASIBLE at the next status
 *                read), mean_out optional; workspace of at least
 *                sdp_split_fleet_workspace_bytes(a, max_routes, route_out !=
 *                NULL) bytes (device, 256-byte aligned).
 *   max_routes:  K, 1..64.
 *   nroutes_out: [S] int32 device or NULL: routes of the optimal split, 0
 *                when infeasible.
 *   route_out:   [S*n] uint8 device or NULL: route_out[s*n + i-1] = index
 *                (0-based, in tour order) of the route serving position i;
 *                0xFF for every position of an infeasible scenario.
 * Errors: SDP_ERR_INVALID_ARG (as sdp_split_eval; pred_out set; host
 * pointers), SDP_ERR_UNSUPPORTED (max_routes outside 1..64, n > 16384,
 * Q > 32767, soft capacity, another algo), SDP_ERR_WORKSPACE. */
size_t sdp_split_fleet_workspace_bytes(const sdp_split_args* a, int32_t max_routes,
                                       int32_t want_routes);
int sdp_split_fleet_eval(const sdp_split_args* a, int32_t max_routes, int32_t* nroutes_out,
                         uint8_t* route_out, void* stream);

/* Number of capacity-feasible arcs (p,i), p < i, load(s_{p+1..i}) <= Q, per
 * scenario -- the relaxations of Eq. eqdpA, the throughput unit.
 * arcs_out [S] int64 or NULL; total_out [1] uint64 (device) or NULL. */
int sdp_split_count_arcs(const sdp_split_args* a, int64_t* arcs_out,
                         uint64_t* total_out, void* stream);

/* Adjoint of the scenario mean of Split with respect to the travel-cost
 * matrix (dist mode only).  The optimal cost is piecewise linear in dist, so
 * at a point where each scenario's optimum is unique
 *     d mean / d dist[a][b] = (1/S) * #uses of arc (a,b) in the optimal routes.
 * fwd: the forward arguments (dist != NULL; cost_out / pred_out / mean_out
 *      are not written).  pred: the forward's predecessors ([S*n], dtype
 *      fwd->pred_dtype) to backtrack, or NULL to recompute them in a fused
 *      forward + backtrack pass that keeps them on chip.
 * grad_mean: [1] device scalar (upstream gradient);
 * grad_dist: [(n+1)*(n+1)] fp32, overwritten with
 *      (count(a,b) / S) * (*grad_mean).
 * route_hist_out: [2n] int64 or NULL: route starts per tour position then
 *      route ends per tour position, summed over feasible scenarios.
 * Infeasible scenarios contribute no arc (the mean is +inf there).
 * Fused pass, default shape (warps_per_cta = 0, ring 0 or 16) and rows that
 * fit the tensor memory (n bytes of uint8 or 2n of uint16 within 512): the
 * deque kernel with TMEM-staged rows and 16 warps per SM (17..24 when that
 * many take every 32-scenario tile in one round where 16 would need two),
 * keeping i - pred(i) in a workspace scratch; otherwise the shared-memory DEQUE kernel keeps them in
 * its staged rows. */
size_t sdp_split_backward_workspace_bytes(const sdp_split_args* fwd);
int sdp_split_backward(const sdp_split_args* fwd, const void* pred,
                       const float* grad_mean, float* grad_dist,
                       int64_t* route_hist_out, void* stream);

/* -------------------------------------------------------- batched Split */
/* The Split of Eq. eqdpA for B giant tours of uneven length, S scenarios
 * each (the candidate evaluations Tables cand_cvrp / gpu_dsirp count), run
 * as one persistent launch (work queue over (tour, 32-scenario tile) items,
 * longest tours first) captured in a CUDA graph.  Offsets are HOST arrays read at plan
 * creation; the device arrays must stay valid while the plan is used. */
typedef struct sdp_split_batch_desc {
  int32_t B;                    /* tours, B >= 1 */
  int32_t Q;                    /* capacity, 1 <= Q <= 32767 */
  int64_t S;                    /* scenarios per tour, S >= 1 */
  const int32_t* n_host;        /* host [B], 1 <= n_b <= 65534 */
  const int64_t* tour_off_host; /* host [B]: tour b = tours[tour_off[b] ..+n_b) */
  const int32_t* tours;         /* device, permutations of 1..n_b */
  const int64_t* coord_off_host;/* host [B]: coords of tour b start at
                                   coords[2*coord_off[b]], (n_b+1) nodes */
  const float* coords;          /* device */
  const int64_t* dem_off_host;  /* host [B]: demands of tour b = [S, n_b]
                                   row-major at demands[dem_off[b]] */
  const int32_t* demands;       /* device */
  float* costs_out;             /* device [B*S], costs_out[b*S + s] */
  double* means_out;            /* device [B] or NULL */
} sdp_split_batch_desc;

typedef struct sdp_plan sdp_plan;
/* Allocates the plan's device memory (offsets, tour records, work counter,
 * fallback list and scratch); SDP_ERR_OOM if that fails.  Uses the current
 * device; every later call on the plan must run with that device current. */
int sdp_split_plan_create(const sdp_split_batch_desc* d, sdp_plan** out);
/* Times the candidate launch shapes (the pipelined and streaming kernels;
 * DEQUE warps per CTA x deque ring entries x scenarios per lane) on
 * `stream` -- each runs the whole plan, so outputs are overwritten -- and
 * keeps the fastest.  cache_path (optional, host string) is a text file of
 * earlier choices keyed by the device and the plan's shape: a hit skips the
 * timing, a miss appends the new choice. */
int sdp_plan_autotune(sdp_plan* p, void* stream, const char* cache_path);
/* Enqueues one evaluation of the whole batch on `stream`: tour preparation,
 * the persistent kernel, the recomputation of the scenarios it flagged (one
 * warp per scenario, the plain kernel's bits) and the per-tour FP64 means.  The first call captures these launches into a CUDA graph;
 * later calls replay it (a new launch shape from autotune re-captures). */
int sdp_plan_run(sdp_plan* p, void* stream);
/* Device time of the persistent kernel in the most recent sdp_plan_run
 * (waits for it). */
int sdp_plan_kernel_ms(sdp_plan* p, float* ms);
/* Launch shape in use and the number of (tour, 32-scenario tile) items.
 * warps_per_cta = -2: the pipelined kernel (SDP_ALGO_PIPE's kernel over the
 * plan's items; chosen when every dem_off is a multiple of 4, demands are
 * 16-byte aligned and n_max <= 1024), -1: the streaming kernel (tiles
 * narrowed into tour order by producer warps; the choice for
 * 1024 < n_max <= 2048 on the same alignment), 0: DEQUE with tensor-memory staging,
 * k > 0: DEQUE with shared-memory staging and k warps per CTA. */
int sdp_plan_info(const sdp_plan* p, int32_t* warps_per_cta, int32_t* ring,
                  int32_t* ctas, int64_t* items);
/* Selects a launch shape by hand (what sdp_plan_autotune chooses among):
 * warps_per_cta -2 (pipelined), -1 (streaming), 0 (DEQUE, tensor-memory
 * staging) or 1..8 (DEQUE, shared-memory staging); ring 8, 16 or 32 deque
 * entries (16 for -2 / -1 / 0); scenarios_per_lane 1, or 2 with
 * shared-memory staging (each lane then runs two scenarios of one tour,
 * their deques stepped together).  The next sdp_plan_run re-captures the
 * graph.  SDP_ERR_UNSUPPORTED (and the plan keeps its shape) when the shape
 * does not apply to this plan or does not fit an SM. */
int sdp_plan_configure(sdp_plan* p, int32_t warps_per_cta, int32_t ring,
                       int32_t scenarios_per_lane);
/* Scenarios per lane of the shape in use (1 or 2). */
int sdp_plan_scenarios_per_lane(const sdp_plan* p, int32_t* scenarios_per_lane);
/* Total feasible arcs of the whole batch (synchronous on `stream`). */
int sdp_plan_count_arcs(sdp_plan* p, void* stream, uint64_t* total_host);
void sdp_plan_destroy(sdp_plan* p);

/* ------------------------------------------------- SAA candidate search */
/* Sample-average-approximation search over first-stage giant tours (the
 * candidate loop of Sec. "Decision Quality under Fixed Time Budgets" and
 * Tables tab:gpu_dsirp / tab:cand_cvrp, where a genetic algorithm proposes
 * candidates and each is scored by the SAA mean of its second-stage Split
 * over the scenario set).  Here a local search proposes them: every
 * iteration evaluates the current tour and B neighbours of it over the same
 * S demand scenarios in one replay of a batched plan (B + 1 tours sharing
 * one demand array and one coordinate array), then moves to the neighbour
 * with the lowest scenario mean if that mean is strictly below the current
 * tour's (ties between neighbours go to the smaller index).  Candidates are
 * built and chosen on the device; the host only enqueues.
 *
 * Neighbour k (0-based) of iteration t draws z = SplitMix64 output number
 * c = t*B + k of the stream `seed` (z = mix(seed + (c+1)*0x9E3779B97F4A7C15),
 * mix = the finaliser of Steele, Lea and Flood's SplittableRandom with
 * Stafford's constants), then
 *     a = (z mod 2^32) mod n,  b = (z >> 40) mod (n-1),  b += (b >= a),
 *     kind = enabled[((z >> 32) & 255) mod #enabled]
 * with the enabled kinds listed in the order 2-opt, relocate, swap:
 *     2-opt:    reverse positions min(a,b) .. max(a,b) of the tour;
 *     relocate: take the customer at position a out and reinsert it so that
 *               it ends at position b;
 *     swap:     exchange the customers at positions a and b.
 * Positions are 0-based indices into the tour array. */
#define SDP_MOVE_2OPT 1
#define SDP_MOVE_RELOCATE 2
#define SDP_MOVE_SWAP 4

typedef struct sdp_saa_search_desc {
  int32_t n;               /* customers, 2 <= n <= 2048 */
  const float* coords;     /* device [(n+1)*2], node 0 = depot */
  int32_t Q;               /* capacity, 1 <= Q <= 32767 */
  int64_t S;               /* scenarios, S >= 1 */
  const int32_t* demands;  /* device [S*n], demands[s*n + (c-1)] = demand of
                              customer c; one scenario set for every candidate */
  int32_t B;               /* neighbours per iteration, 1 <= B <= 2^20 */
  uint64_t seed;           /* move stream */
  int32_t moves;           /* nonzero OR of SDP_MOVE_* */
  const int32_t* tour0;    /* device [n]: the starting tour, a permutation of
                              1..n (copied at create) */
} sdp_saa_search_desc;

typedef struct sdp_saa_search sdp_saa_search;
/* Allocates the search (its batched plan, B + 1 candidate tours, their costs
 * and means, the current tour); SDP_ERR_OOM if that fails.  Errors:
 * SDP_ERR_INVALID_ARG for a NULL desc / out, B, S or moves out of range, or
 * coords / demands / tour0 not in device memory; SDP_ERR_UNSUPPORTED for n
 * outside 2..2048 or Q outside 1..32767.  tour0 is not checked here: a
 * customer id outside 1..n is read as customer 1 and raises
 * SDP_FLAG_DEVICE_CHECK in the status word at the first run (a repeated id
 * is not detected and scores a different tour).  The caller's
 * coords and demands must stay valid until destroy.  Uses the current
 * device; later calls must run with that device current (run and state
 * return SDP_ERR_INVALID_ARG otherwise, launching nothing).  A search is used
 * from one thread at a time (like a plan); its calls are ordered on the
 * stream they are given. */
int sdp_saa_search_create(const sdp_saa_search_desc* d, sdp_saa_search** out);
/* Runs `iters` iterations on `stream` (continuing the move stream where the
 * previous run stopped).  trace_out: device [iters] fp64 or NULL: the best
 * mean after each iteration; accepted_out: device [iters] int32 or NULL: the
 * neighbour taken (0..B-1), or -1 if none improved. */
int sdp_saa_search_run(sdp_saa_search* s, int32_t iters, double* trace_out,
                       int32_t* accepted_out, void* stream);
/* Current tour (device [n] int32) and, if means_out (device [B+1] fp64) is
 * set, the means of the last iteration: [0] the tour it started from, [1+k]
 * neighbour k.  Before any iteration the means are not defined. */
int sdp_saa_search_state(sdp_saa_search* s, int32_t* tour_out, double* means_out,
                         void* stream);
/* Capacity-feasible arcs (p, i) of Eq. eqdpA summed over the scenarios of
 * every tour the last iteration scored (the current tour and its B
 * neighbours), as sdp_plan_count_arcs: the throughput unit of the search.
 * total_out: host uint64; synchronises `stream`. */
int sdp_saa_search_count_arcs(sdp_saa_search* s, void* stream, uint64_t* total_out);
/* sizeof(sdp_saa_search_desc) as compiled into the library (binding checks). */
size_t sdp_saa_search_desc_size(void);
/* sdp_plan_autotune on the search's plan, deque rings of 16 entries only:
 * the tours change as the search goes, and a ring sized on the first ones can
 * overflow on later, better tours (longer monotone runs in the deque), whose
 * scenarios then go to the plain fallback.  Overwrites the last means. */
int sdp_saa_search_autotune(sdp_saa_search* s, void* stream, const char* cache_path);
/* Launch shape of the search's plan (as sdp_plan_info and
 * sdp_plan_scenarios_per_lane report it for a plan; any pointer may be NULL).
 * Host-side only.  Errors: SDP_ERR_INVALID_ARG (s NULL). */
int sdp_saa_search_plan_info(const sdp_saa_search* s, int32_t* warps_per_cta, int32_t* ring,
                             int32_t* ctas, int32_t* scenarios_per_lane);
void sdp_saa_search_destroy(sdp_saa_search* s);

/* ------------------------------------------------------------ Reinsertion */
/* One customer, order-up-to level U, days t = 0..T-1, S scenarios.
 * State: start-of-day inventory I in 0..U.  Actions q in {0, U-I}; delivery
 * arrives before consumption; unmet demand is lost:
 *     I' = max(0, I + q - d_t).
 * Stage cost F_t(q) + e(I + q - d_t) with F_t(q) = fixed[t] + unit_cost*q for
 * q > 0 and 0 for q = 0; e(x) = h*x for x >= 0 and p*(-x) for x < 0, or, if
 * end_cost_table != NULL, e(x) = end_cost_table[max(0,x)].  Terminal cost 0.
 * Backward DP C_T = 0, C_t(I) = min(no delivery, delivery), ties to no
 * delivery; value = C_0(I0); policy = decisions along the optimal path. */
/* Reinsertion kernels */
#define SDP_REINSERT_AUTO 0  /* LANE where it applies (measured faster at
                                T = 60, U = 200, with and without route
                                options), else WARP */
#define SDP_REINSERT_WARP 1  /* one warp per scenario, states across lanes */
#define SDP_REINSERT_LANE 2  /* one lane per scenario, its cost-to-go in shared
                                memory (up to 8 warps per SM); needs U <= 255;
                                with a policy, its decision bits take
                                workspace (SMs x 8 x T x ceil((U+1)/32) x 128
                                bytes) */
typedef struct sdp_reinsert_args {
  int32_t T;                  /* 1 <= T; T * W <= 4096 where W = 8 for
                                 U < 256, 16 for U < 512, 32 for U < 1024
                                 (decision bits stay on chip), else
                                 SDP_ERR_UNSUPPORTED */
  int32_t U;                  /* 0 <= U <= 1023 */
  int32_t I0;                 /* 0 <= I0 <= U */
  int32_t algo;               /* SDP_REINSERT_AUTO / _WARP / _LANE */
  float h, p, unit_cost;
  int64_t S;                  /* scenarios, S >= 0 */
  const float* fixed;         /* [T] per-day routing/insertion cost f_t */
  const float* end_cost_table;/* [U+1] or NULL */
  const int32_t* consumption; /* [S*T], consumption[s*T + t] */
  float* value_out;           /* [S], required */
  uint8_t* policy_out;        /* [S*T] or NULL: 1 = deliver up to U on day t */
  float* value0_out;          /* [S*(U+1)] or NULL: C_0(I) for every I */
  double* mean_out;           /* [1] or NULL */
  void* workspace;
  size_t workspace_bytes;
  int32_t n_routes;           /* K route options per day (0: the single route
                                 of `fixed`).  With K > 0 a delivery of
                                 q = U - I on day t may ride route r only if
                                 route_cap[(s*T + t)*K + r] >= q, at cost
                                 route_cost[t*K + r] (+ unit_cost * q); the
                                 cheapest such route is taken, none -> no
                                 delivery (an entry of the transition matrix
                                 is a minimum over route options, Sec. 2
                                 "Instantiation B").  policy_out then holds
                                 0 (no delivery) or r + 1; `fixed` is not
                                 read.  Needs U <= 255, K <= 64, no
                                 end_cost_table; LANE takes K <= 8 (the
                                 same bits as WARP), AUTO takes LANE there
                                 and WARP beyond. */
  const float* route_cost;    /* [T*K] */
  const int32_t* route_cap;   /* [S*T*K] */
} sdp_reinsert_args;

size_t sdp_reinsert_args_size(void);
size_t sdp_reinsert_workspace_bytes(const sdp_reinsert_args* a);
int sdp_reinsert_eval(const sdp_reinsert_args* a, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SDP_H_ */

// saa_search.cu -- sample-average-approximation search over first-stage
// giant tours.  Every iteration scores the current tour and B neighbours of it
// by their Split mean over one scenario set (the candidate loop of the
// paper's fixed-time-budget experiments, Tables tab:gpu_dsirp /
// tab:cand_cvrp), in one replay of a batched plan of B + 1 tours that share
// the demand and coordinate arrays, and moves to the best neighbour when its
// mean is strictly lower.  All of it stays on the device:
//   saa_candidates_kernel  block k writes tour k of the plan (k = 0: the
//                          current tour; k >= 1: move k - 1 applied to it),
//   plan replay            tour prep, persistent Split kernel, FP64 means,
//   saa_select_kernel      argmin over the neighbours, acceptance, trace.
// The moves come from a counter-based generator (SplitMix64) so that any
// iteration's candidates can be rebuilt from (seed, iteration, index).
#include <stdio.h>

#include <vector>

#include <math_constants.h>

#include "sdp_internal.cuh"

struct sdp_saa_search {
  int device = 0;
  int n = 0, B = 0, moves = 0;
  int64_t S = 0;
  int64_t iter = 0;  // iterations run so far: the move stream's position
  uint64_t seed = 0;
  sdp_plan* plan = nullptr;
  int32_t* d_cand = nullptr;   // [(B+1) * n] the plan's tours
  float* d_costs = nullptr;    // [(B+1) * S]
  double* d_means = nullptr;   // [B+1]
  int32_t* d_cur = nullptr;    // [n] current tour
};

namespace sdp {
int api_fail(int code, const char* msg);  // sdp_api.cu
bool api_device_ptr(const void* p);      // sdp_api.cu
int plan_autotune(sdp_plan* p, void* stream, const char* cache_path, int min_ring);  // split_batch.cu
namespace {

bool is_device_ptr(const void* p) { return api_device_ptr(p); }

// The search's buffers and the caller's stream belong to the device that was
// current at creation; run and state need it current again.
bool on_own_device(const sdp_saa_search* s) {
  int d = -1;
  return cudaGetDevice(&d) == cudaSuccess && d == s->device;
}

int sfail(int code, const char* msg) { return api_fail(code, msg); }

int scuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return api_fail(SDP_ERR_CUDA, buf);
}

// SplitMix64 output number c of the stream seeded with `seed`: the state
// after c + 1 Weyl increments, through the 64-bit finaliser.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Move {
  int kind;  // 0 = 2-opt, 1 = relocate, 2 = swap
  int a, b;  // 2-opt: a < b
};

__device__ __forceinline__ Move decode_move(uint64_t z, int n, int mask) {
  int kinds[3];
  int nk = 0;
  if (mask & SDP_MOVE_2OPT) kinds[nk++] = 0;
  if (mask & SDP_MOVE_RELOCATE) kinds[nk++] = 1;
  if (mask & SDP_MOVE_SWAP) kinds[nk++] = 2;
  const int a = (int)((uint32_t)z % (uint32_t)n);
  int b = (int)((uint32_t)(z >> 40) % (uint32_t)(n - 1));
  if (b >= a) ++b;
  Move m;
  m.kind = kinds[(uint32_t)((z >> 32) & 0xFFu) % (uint32_t)nk];
  m.a = (m.kind == 0) ? min(a, b) : a;
  m.b = (m.kind == 0) ? max(a, b) : b;
  return m;
}

// Position of the current tour that lands at position m of the neighbour.
__device__ __forceinline__ int move_source(const Move& mv, int m) {
  const int a = mv.a, b = mv.b;
  if (mv.kind == 0) return (m >= a && m <= b) ? a + b - m : m;
  if (mv.kind == 1) {
    if (m == b) return a;
    if (a < b) return (m >= a && m < b) ? m + 1 : m;
    return (m > b && m <= a) ? m - 1 : m;
  }
  return m == a ? b : (m == b ? a : m);
}

// Block k: tour k of the plan.  k = 0 copies the current tour, k >= 1 applies
// move number iter * B + (k - 1).
__global__ void saa_candidates_kernel(const int32_t* __restrict__ cur, int32_t* __restrict__ cand,
                                      int n, int B, uint64_t seed, int64_t iter, int mask) {
  const int k = blockIdx.x;
  int32_t* out = cand + (int64_t)k * n;
  if (k == 0) {
    for (int m = threadIdx.x; m < n; m += blockDim.x) out[m] = cur[m];
    return;
  }
  const uint64_t c = (uint64_t)iter * (uint64_t)B + (uint64_t)(k - 1);
  const Move mv = decode_move(splitmix64(seed, c), n, mask);
  for (int m = threadIdx.x; m < n; m += blockDim.x) out[m] = cur[move_source(mv, m)];
}

// Block k: a copy of tour t into slot k.
__global__ void saa_fill_kernel(const int32_t* __restrict__ t, int32_t* __restrict__ cand, int n) {
  int32_t* out = cand + (int64_t)blockIdx.x * n;
  for (int m = threadIdx.x; m < n; m += blockDim.x) out[m] = t[m];
}

// One block: the neighbour with the lowest mean (a NaN never wins; ties go to
// the smaller index) replaces the current tour if its mean is strictly below
// the current tour's (means[0]).
constexpr int kSelectThreads = 1024;
__global__ void __launch_bounds__(kSelectThreads) saa_select_kernel(
    const double* __restrict__ means, int B, const int32_t* __restrict__ cand, int n,
    int32_t* __restrict__ cur, double* trace, int32_t* accepted, int t) {
  __shared__ double sv[kSelectThreads / 32];
  __shared__ int sk[kSelectThreads / 32];
  __shared__ int win;
  double v = CUDART_INF;
  int kk = B;
  for (int k = threadIdx.x; k < B; k += blockDim.x) {
    const double m = means[1 + k];
    if (m < v) {  // k grows within a thread: the first minimum stays
      v = m;
      kk = k;
    }
  }
  auto better = [](double v1, int k1, double v2, int k2) {
    return v2 < v1 || (v2 == v1 && k2 < k1);
  };
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int k2 = __shfl_down_sync(0xffffffffu, kk, o);
    if (better(v, kk, v2, k2)) {
      v = v2;
      kk = k2;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sv[warp] = v;
    sk[warp] = kk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (better(v, kk, sv[w], sk[w])) {
        v = sv[w];
        kk = sk[w];
      }
    const double m0 = means[0];
    const bool take = kk < B && v < m0;
    win = take ? kk : -1;
    if (trace) trace[t] = take ? v : m0;
    if (accepted) accepted[t] = win;
  }
  __syncthreads();
  if (win >= 0) {
    const int32_t* src = cand + (int64_t)(1 + win) * n;
    for (int m = threadIdx.x; m < n; m += blockDim.x) cur[m] = src[m];
  }
}

}  // namespace
}  // namespace sdp

using namespace sdp;

extern "C" {

void sdp_saa_search_destroy(sdp_saa_search* s) {
  if (!s) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  sdp_plan_destroy(s->plan);
  cudaFree(s->d_cand);
  cudaFree(s->d_costs);
  cudaFree(s->d_means);
  cudaFree(s->d_cur);
  cudaSetDevice(prev);
  delete s;
}

int sdp_saa_search_create(const sdp_saa_search_desc* d, sdp_saa_search** out) {
  if (!d || !out) return sfail(SDP_ERR_INVALID_ARG, "desc / out is NULL");
  *out = nullptr;
  if (d->n < 2 || d->n > 2048) return sfail(SDP_ERR_UNSUPPORTED, "search needs 2 <= n <= 2048");
  if (d->B < 1 || d->B > (1 << 20)) return sfail(SDP_ERR_INVALID_ARG, "B outside 1..2^20");
  if (d->S < 1) return sfail(SDP_ERR_INVALID_ARG, "S < 1");
  if (d->moves == 0 || (d->moves & ~(SDP_MOVE_2OPT | SDP_MOVE_RELOCATE | SDP_MOVE_SWAP)))
    return sfail(SDP_ERR_INVALID_ARG, "moves must be a nonzero OR of SDP_MOVE_*");
  if (!is_device_ptr(d->coords) || !is_device_ptr(d->demands) || !is_device_ptr(d->tour0))
    return sfail(SDP_ERR_INVALID_ARG, "coords / demands / tour0 must be device pointers");
  auto* s = new sdp_saa_search();
  cudaGetDevice(&s->device);
  s->n = d->n;
  s->B = d->B;
  s->S = d->S;
  s->moves = d->moves;
  s->seed = d->seed;
  const int T = d->B + 1;
  cudaError_t e = fault_alloc() ? cudaErrorMemoryAllocation  // injected (tests)
                                : cudaMalloc((void**)&s->d_cand, sizeof(int32_t) * (size_t)T * d->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_costs, sizeof(float) * (size_t)T * d->S);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_means, sizeof(double) * (size_t)T);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_cur, sizeof(int32_t) * (size_t)d->n);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_cur, d->tour0, sizeof(int32_t) * (size_t)d->n, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) {  // every slot holds a valid tour before the first replay
    saa_fill_kernel<<<T, 128>>>(s->d_cur, s->d_cand, d->n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    sdp_saa_search_destroy(s);
    return e == cudaErrorMemoryAllocation ? sfail(SDP_ERR_OOM, "search allocation failed")
                                          : scuda(e, "search create");
  }
  std::vector<int32_t> nh(T, d->n);
  std::vector<int64_t> toff(T), zero(T, 0);
  for (int k = 0; k < T; ++k) toff[k] = (int64_t)k * d->n;
  sdp_split_batch_desc bd{};
  bd.B = T;
  bd.Q = d->Q;
  bd.S = d->S;
  bd.n_host = nh.data();
  bd.tour_off_host = toff.data();
  bd.tours = s->d_cand;
  bd.coord_off_host = zero.data();
  bd.coords = d->coords;
  bd.dem_off_host = zero.data();
  bd.demands = d->demands;
  bd.costs_out = s->d_costs;
  bd.means_out = s->d_means;
  const int rc = sdp_split_plan_create(&bd, &s->plan);
  if (rc) {
    sdp_saa_search_destroy(s);
    return rc;
  }
  *out = s;
  return SDP_OK;
}

int sdp_saa_search_run(sdp_saa_search* s, int32_t iters, double* trace_out,
                       int32_t* accepted_out, void* stream) {
  if (!s) return sfail(SDP_ERR_INVALID_ARG, "search is NULL");
  if (!on_own_device(s)) return sfail(SDP_ERR_INVALID_ARG, "the search's device is not current");
  if (iters < 0) return sfail(SDP_ERR_INVALID_ARG, "iters < 0");
  if (trace_out && !is_device_ptr(trace_out))
    return sfail(SDP_ERR_INVALID_ARG, "trace_out must be a device pointer");
  if (accepted_out && !is_device_ptr(accepted_out))
    return sfail(SDP_ERR_INVALID_ARG, "accepted_out must be a device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int t = 0; t < iters; ++t) {
    saa_candidates_kernel<<<s->B + 1, 128, 0, st>>>(s->d_cur, s->d_cand, s->n, s->B, s->seed,
                                                    s->iter, s->moves);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(e, "search candidates");
    const int rc = sdp_plan_run(s->plan, stream);
    if (rc) return rc;
    saa_select_kernel<<<1, kSelectThreads, 0, st>>>(s->d_means, s->B, s->d_cand, s->n, s->d_cur,
                                                     trace_out, accepted_out, t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(e, "search select");
    ++s->iter;
  }
  return SDP_OK;
}

int sdp_saa_search_state(sdp_saa_search* s, int32_t* tour_out, double* means_out,
                         void* stream) {
  if (!s) return sfail(SDP_ERR_INVALID_ARG, "search is NULL");
  if (!on_own_device(s)) return sfail(SDP_ERR_INVALID_ARG, "the search's device is not current");
  if (!tour_out || !is_device_ptr(tour_out))
    return sfail(SDP_ERR_INVALID_ARG, "tour_out must be a device pointer");
  if (means_out && !is_device_ptr(means_out))
    return sfail(SDP_ERR_INVALID_ARG, "means_out must be a device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(tour_out, s->d_cur, sizeof(int32_t) * (size_t)s->n,
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && means_out)
    e = cudaMemcpyAsync(means_out, s->d_means, sizeof(double) * (size_t)(s->B + 1),
                        cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return scuda(e, "search state");
  return SDP_OK;
}

int sdp_saa_search_count_arcs(sdp_saa_search* s, void* stream, uint64_t* total_out) {
  if (!s) return sfail(SDP_ERR_INVALID_ARG, "search is NULL");
  if (!on_own_device(s)) return sfail(SDP_ERR_INVALID_ARG, "the search's device is not current");
  return sdp_plan_count_arcs(s->plan, stream, total_out);
}

size_t sdp_saa_search_desc_size(void) { return sizeof(sdp_saa_search_desc); }

int sdp_saa_search_autotune(sdp_saa_search* s, void* stream, const char* cache_path) {
  if (!s) return sfail(SDP_ERR_INVALID_ARG, "search is NULL");
  return plan_autotune(s->plan, stream, cache_path, 16);
}

int sdp_saa_search_plan_info(const sdp_saa_search* s, int32_t* warps_per_cta, int32_t* ring,
                             int32_t* ctas, int32_t* scenarios_per_lane) {
  if (!s) return sfail(SDP_ERR_INVALID_ARG, "search is NULL");
  const int rc = sdp_plan_info(s->plan, warps_per_cta, ring, ctas, nullptr);
  if (rc) return rc;
  return scenarios_per_lane ? sdp_plan_scenarios_per_lane(s->plan, scenarios_per_lane) : SDP_OK;
}

}  // extern "C"

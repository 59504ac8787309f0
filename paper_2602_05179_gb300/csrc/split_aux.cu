// split_aux.cu -- tour preparation, feasible-arc counting, the deterministic
// FP64 scenario mean, and the Split adjoint's backtrack / gradient assembly.
#include "sdp_internal.cuh"

namespace sdp {

// Travel cost c(a,b).  Coordinates: FP32 Euclidean distance with IEEE
// rounding at every step (no contraction, correctly rounded sqrt), so every
// launch and every kernel sees the same bits.  Matrix: dist[a*(n+1)+b].
__device__ __forceinline__ float travel(const float* coords, const float* dist,
                                        int n, int a, int b) {
  if (dist) return __ldg(dist + (size_t)a * (n + 1) + b);
  float dx = __fsub_rn(__ldg(coords + 2 * a), __ldg(coords + 2 * b));
  float dy = __fsub_rn(__ldg(coords + 2 * a + 1), __ldg(coords + 2 * b + 1));
  return __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
}

// One CTA per tour (Sec. 2 Instantiation A: the route cost W(p,i) depends on
// the tour only through c(0,s_{p+1}), the consecutive arcs and c(s_i,0)).
__global__ void __launch_bounds__(256) tour_prep_kernel(
    const int32_t* __restrict__ tour, int n, const float* __restrict__ coords,
    const float* __restrict__ dist, TourPrep prep, uint32_t* status,
    uint32_t* reset_word) {
  __shared__ double red[256];
  if (threadIdx.x == 0 && reset_word) *reset_word = 0u;
  double acc = 0.0;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int si = __ldg(tour + i);
    if (si < 1 || si > n) { bad = true; si = 1; }
    float c0 = travel(coords, dist, n, 0, si);
    float ce = travel(coords, dist, n, si, 0);
    float e = 0.f;
    if (i > 0) {
      int sp = __ldg(tour + i - 1);
      if (sp < 1 || sp > n) sp = 1;
      e = travel(coords, dist, n, sp, si);
      acc += (double)e;  // D(n) = sum of the n-1 consecutive arcs
    }
    StepRec r;
    r.col = (uint32_t)(si - 1);
    r.a = __fsub_rn(c0, e);
    r.ce = ce;
    r.pad = 0u;
    prep.rec[i] = r;
    prep.cols[i] = (uint16_t)(si - 1);
  }
  if (bad) atomicOr(status, SDP_FLAG_DEVICE_CHECK);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *prep.Dn = red[0];
}

void launch_tour_prep(const int32_t* tour, int n, const float* coords,
                      const float* dist, TourPrep prep, uint32_t* status,
                      uint32_t* reset_word, cudaStream_t st) {
  tour_prep_kernel<<<1, 256, 0, st>>>(tour, n, coords, dist, prep, status,
                                      reset_word);
}

// ----------------------------------------------------------- arc counting
// Feasible arcs of scenario s: sum_i (i - pmin(i)), pmin(i) the smallest p
// with load(s_{p+1..i}) <= Q (two pointers; the load is monotone).
__global__ void __launch_bounds__(256) count_arcs_kernel(
    int n, int Q, int64_t S, const StepRec* __restrict__ rec,
    const int32_t* __restrict__ demands, int64_t* __restrict__ arcs,
    unsigned long long* total) {
  unsigned long long mine = 0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* q = demands + s * n;
    int64_t W = 0, cnt = 0;
    int pm = 0;
    for (int i = 1; i <= n; ++i) {
      W += max(__ldg(q + __ldg(&rec[i - 1].col)), 0);
      while (W > Q && pm < i) {
        ++pm;
        W -= max(__ldg(q + __ldg(&rec[pm - 1].col)), 0);
      }
      cnt += i - pm;
    }
    if (arcs) arcs[s] = cnt;
    mine += (unsigned long long)cnt;
  }
  if (total) {
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
  }
}

void launch_count_arcs(int n, int Q, int64_t S, const StepRec* rec,
                       const int32_t* demands, int64_t* arcs,
                       unsigned long long* total, int grid, cudaStream_t st) {
  count_arcs_kernel<<<grid, 256, 0, st>>>(n, Q, S, rec, demands, arcs, total);
}

// ------------------------------------------------------------- FP64 mean
// Two passes with a fixed blocking: block b sums its contiguous chunk with a
// fixed per-thread order and a fixed tree, then one block sums the partials.
// The result does not depend on scheduling (bit-reproducible).
__global__ void __launch_bounds__(256) mean_partial_kernel(
    const float* __restrict__ x, int64_t count, double* partial) {
  __shared__ double red[256];
  const int64_t chunk = (count + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(count, lo + chunk);
  double acc = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) acc += (double)x[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kMeanBlocks) mean_final_kernel(
    const double* __restrict__ partial, int64_t count, double* out) {
  __shared__ double red[kMeanBlocks];
  red[threadIdx.x] = partial[threadIdx.x];
  __syncthreads();
  for (int w = kMeanBlocks / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = count > 0 ? red[0] / (double)count : 0.0;
}

void launch_mean(const float* x, int64_t count, double* partial, double* out,
                 cudaStream_t st) {
  mean_partial_kernel<<<kMeanBlocks, 256, 0, st>>>(x, count, partial);
  mean_final_kernel<<<1, kMeanBlocks, 0, st>>>(partial, count, out);
}

// ------------------------------------------------------------------ adjoint
// Backtrack of stored predecessors: for each scenario walk i = n -> pred(i)
// -> ... -> 0; route p+1..i starts at position p+1 and ends at position i.
// hist[0..n) = starts, hist[n..2n) = ends, hist[2n] = scenarios counted.
template <typename PT>
__global__ void __launch_bounds__(256) backtrack_hist_kernel(
    int n, int64_t S, const PT* __restrict__ pred,
    unsigned long long* __restrict__ hist, uint32_t* status) {
  extern __shared__ unsigned int sh[];
  const bool use_smem = (2 * n + 1) * 4 <= 48 * 1024;
  if (use_smem)
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x) sh[k] = 0u;
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const PT* ps = pred + s * n;
    bool ok = true;
    for (int i = n; i > 0;) {
      long long p = (long long)ps[i - 1];
      if (sizeof(PT) == 2 && p == 0xFFFF) p = -1;
      if (p < 0 || p >= i) { ok = false; break; }
      i = (int)p;
    }
    if (!ok) continue;
    for (int i = n; i > 0;) {
      int p = (int)ps[i - 1];
      if (use_smem) {
        atomicAdd(&sh[p], 1u);
        atomicAdd(&sh[n + i - 1], 1u);
      } else {
        atomicAdd(&hist[p], 1ull);
        atomicAdd(&hist[n + i - 1], 1ull);
      }
      i = p;
    }
    if (use_smem) atomicAdd(&sh[2 * n], 1u);
    else atomicAdd(&hist[2 * n], 1ull);
  }
  __syncthreads();
  if (use_smem)
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x)
      if (sh[k]) atomicAdd(&hist[k], (unsigned long long)sh[k]);
}

void launch_backtrack_hist(int n, int64_t S, const void* pred, int pred_dtype,
                           unsigned long long* hist, uint32_t* status,
                           cudaStream_t st) {
  int grid = 2 * num_sms();
  size_t smem = (2 * (size_t)n + 1) * 4 <= 48 * 1024 ? (2 * (size_t)n + 1) * 4 : 0;
  if (pred_dtype == SDP_PRED_U16)
    backtrack_hist_kernel<uint16_t><<<grid, 256, smem, st>>>(
        n, S, (const uint16_t*)pred, hist, status);
  else
    backtrack_hist_kernel<int32_t><<<grid, 256, smem, st>>>(
        n, S, (const int32_t*)pred, hist, status);
}

__global__ void zero_kernel(float* g, int64_t count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x)
    g[k] = 0.f;
}

// Each route p+1..i uses (0,s_{p+1}), (s_k,s_{k+1}) for p+1 <= k < i and
// (s_i,0).  Position k either ends its route (arc (s_k,0)) or continues to
// s_{k+1}: continue(k) = counted scenarios - ends(k).  The arcs touched by
// different positions are distinct because the tour is a permutation.
__global__ void grad_scatter_kernel(int n, int64_t S, const int32_t* __restrict__ tour,
                                    const unsigned long long* __restrict__ hist,
                                    const float* __restrict__ grad_mean,
                                    float* __restrict__ grad, int64_t* hist_out) {
  const double scale = (double)__ldg(grad_mean) / (double)S;
  const unsigned long long used = hist[2 * n];
  const int m = n + 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += gridDim.x * blockDim.x) {
    int sk = __ldg(tour + k);
    if (sk < 1 || sk > n) continue;  // invalid tour entry (flagged by tour_prep)
    unsigned long long st = hist[k], en = hist[n + k];
    grad[(size_t)0 * m + sk] = (float)((double)st * scale);
    grad[(size_t)sk * m + 0] = (float)((double)en * scale);
    if (k + 1 < n) {
      int sn = __ldg(tour + k + 1);
      if (sn >= 1 && sn <= n) grad[(size_t)sk * m + sn] = (float)((double)(used - en) * scale);
    }
    if (hist_out) {
      hist_out[k] = (int64_t)st;
      hist_out[n + k] = (int64_t)en;
    }
  }
}

void launch_grad_assemble(int n, int64_t S, const int32_t* tour,
                          const unsigned long long* hist, const float* grad_mean,
                          float* grad, int64_t* hist_out, cudaStream_t st) {
  int64_t cnt = (int64_t)(n + 1) * (n + 1);
  int g1 = (int)imin64((cnt + 255) / 256, 4 * num_sms());
  zero_kernel<<<g1, 256, 0, st>>>(grad, cnt);
  if (n > 0 && S > 0) {
    int g2 = (n + 255) / 256;
    grad_scatter_kernel<<<g2, 256, 0, st>>>(n, S, tour, hist, grad_mean, grad,
                                            hist_out);
  }
}

}  // namespace sdp

namespace sdp {

// ------------------------------------------------------------ batched Split
// Tour prep for every tour of a batch: one CTA per tour, same arithmetic as
// tour_prep_kernel.
__global__ void __launch_bounds__(256) batch_prep_kernel(BatchPrepArgs a) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  const int n = a.n[b];
  const int32_t* tour = a.tours + a.tour_off[b];
  const float* coords = a.coords + 2 * a.coord_off[b];
  StepRec* rec = a.rec + a.rec_off[b];
  if (b == 0 && threadIdx.x == 0) {
    *a.counter = 0ull;
    *a.fb_count = 0u;
  }
  double acc = 0.0;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int si = __ldg(tour + i);
    if (si < 1 || si > n) { bad = true; si = 1; }
    const float c0 = travel(coords, nullptr, n, 0, si);
    const float ce = travel(coords, nullptr, n, si, 0);
    float e = 0.f;
    if (i > 0) {
      int sp = __ldg(tour + i - 1);
      if (sp < 1 || sp > n) sp = 1;
      e = travel(coords, nullptr, n, sp, si);
      acc += (double)e;
    }
    StepRec r;
    r.col = (uint32_t)(si - 1);
    r.a = __fsub_rn(c0, e);
    r.ce = ce;
    r.pad = 0u;
    rec[i] = r;
  }
  if (bad) atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.Dn[b] = red[0];
}

void launch_batch_prep(const BatchPrepArgs& a, int B, cudaStream_t st) {
  batch_prep_kernel<<<B, 256, 0, st>>>(a);
}

// Per-tour FP64 mean of costs[b*S .. b*S+S): one CTA per tour, fixed order.
__global__ void __launch_bounds__(256) batch_mean_kernel(const float* __restrict__ costs,
                                                         int64_t S, double* means) {
  __shared__ double red[256];
  const float* x = costs + (int64_t)blockIdx.x * S;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < S; k += blockDim.x) acc += (double)x[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) means[blockIdx.x] = red[0] / (double)S;
}

void launch_batch_means(const float* costs, int B, int64_t S, double* means, cudaStream_t st) {
  batch_mean_kernel<<<B, 256, 0, st>>>(costs, S, means);
}

// Feasible arcs of every (tour, scenario) of a batch.
__global__ void __launch_bounds__(256) batch_count_kernel(BatchPrepArgs a, int B, int64_t S,
                                                          int Q, const int64_t* dem_off,
                                                          const int32_t* demands,
                                                          unsigned long long* total) {
  unsigned long long mine = 0;
  const int64_t N = (int64_t)B * S;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(g / S);
    const int64_t s = g - (int64_t)b * S;
    const int n = a.n[b];
    const StepRec* rec = a.rec + a.rec_off[b];
    const int32_t* q = demands + dem_off[b] + s * n;
    int64_t W = 0, cnt = 0;
    int pm = 0;
    for (int i = 1; i <= n; ++i) {
      W += max(__ldg(q + __ldg(&rec[i - 1].col)), 0);
      while (W > Q && pm < i) {
        ++pm;
        W -= max(__ldg(q + __ldg(&rec[pm - 1].col)), 0);
      }
      cnt += i - pm;
    }
    mine += (unsigned long long)cnt;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
}

void launch_batch_count(const BatchPrepArgs& a, int B, int64_t S, int Q, const int64_t* dem_off,
                        const int32_t* demands, unsigned long long* total, cudaStream_t st) {
  batch_count_kernel<<<8 * num_sms(), 256, 0, st>>>(a, B, S, Q, dem_off, demands, total);
}

}  // namespace sdp

// split_rescue.cu -- recomputation of the scenarios a deque kernel flagged
// (its deque outgrew the ring), one warp per scenario, for sm_103a.
//
// Eq. eqdpA in the K-form of sdp_internal.cuh: K(i) = min over the
// capacity-feasible p < i of K(p) + a_{p+1}, plus ce_i.  The candidates of
// position i are spread over the lanes, p = i - 1 - lane - 32 c for chunks
// c = 0, 1, ..., until a chunk meets an infeasible p (the route load only
// grows as p falls, so every smaller p is infeasible too); a butterfly
// reduction takes the minimum, ties to the smallest p (reading S4).  The
// scenario's prefix loads L and its K values sit in shared memory, [n+1] of
// each per warp, so a step costs a few shared-memory reads and five shuffle
// rounds where the one-thread-per-scenario plain kernel paid a chain of
// dependent global loads per arc (milliseconds for a handful of flagged
// scenarios at n = 1000).  The FP32 arithmetic is the plain kernel's,
// operation for operation (psi = K(p) + a_{p+1} rounded, the minimum, then
// + ce_i rounded), so the results are the same bits whichever kernel ran.
// Demands are clamped to [0, Q+1]: a route holding a demand above Q is
// infeasible whatever its value, and the prefix loads stay below 2^31.
#include <math_constants.h>

#include <algorithm>

#include "sdp_internal.cuh"

namespace sdp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRescueMaxWarps = 8;                 // warps per CTA
constexpr size_t kRescueCtaBudget = 96u * 1024u;   // shared memory per CTA we aim for
constexpr size_t kRescueWarpMax = 200u * 1024u;    // one warp's [n+1] K and L at most

size_t rescue_per_warp(int n_max) { return (size_t)2 * sizeof(float) * ((size_t)n_max + 1); }

template <typename PT, bool BATCH>
__global__ void __launch_bounds__(kRescueMaxWarps * 32) split_rescue_kernel(RescueArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)a.n_max + 1;
  float* Ks = reinterpret_cast<float*>(smem) + (int64_t)wib * 2 * stride;
  int32_t* Ls = reinterpret_cast<int32_t*>(Ks + stride);
  const int Q = a.Q;
  const int64_t nwork = (int64_t)(*a.fb_count);
  const int64_t nw = (int64_t)gridDim.x * wpb;
  bool neg = false, inf_any = false;
  for (int64_t w = (int64_t)blockIdx.x * wpb + wib; w < nwork; w += nw) {
    int n;
    const StepRec* rec;
    const int32_t* q;
    double Dn;
    int64_t out;
    if (BATCH) {
      const unsigned long long g = a.fb_list[w];
      const int b = (int)(g / (unsigned long long)a.S);
      const int64_t s = (int64_t)(g - (unsigned long long)b * (unsigned long long)a.S);
      n = a.n[b];
      rec = a.rec + a.rec_off[b];
      q = a.demands + a.dem_off[b] + s * n;
      Dn = a.Dn[b];
      out = (int64_t)g;
    } else {
      const int64_t s = (int64_t)a.fb_list1[w];
      n = a.n1;
      rec = a.rec;
      q = a.demands + s * n;
      Dn = n > 0 ? *a.Dn : 0.0;
      out = s;
    }
    __syncwarp();  // the previous scenario's reads of Ks / Ls are done
    // prefix loads L(i) = q(s_1) + ... + q(s_i), 32 positions per round
    int carry = 0;
    if (lane == 0) Ls[0] = 0;
    for (int i0 = 1; i0 <= n; i0 += 32) {
      const int i = i0 + lane;
      int v = 0;
      if (i <= n) {
        const int raw = __ldg(q + __ldg(&rec[i - 1].col));
        neg |= raw < 0;
        v = min(max(raw, 0), Q + 1);
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += t;
      }
      if (i <= n) Ls[i] = carry + v;
      carry += __shfl_sync(kFull, v, 31);
    }
    if (lane == 0) Ks[0] = 0.f;
    __syncwarp();
    PT* pr = (!BATCH && a.pred) ? reinterpret_cast<PT*>(a.pred) + out * n : nullptr;
    float K = 0.f;
    int pv = -1;  // lane k keeps the predecessor of position (block start) + k
    for (int i = 1; i <= n; ++i) {
      const int Li = Ls[i];
      float best = CUDART_INF_F;
      int bp = 0x7FFFFFFF;
      for (int p = i - 1 - lane;; p -= 32) {
        const bool ok = p >= 0 && Li - Ls[p] <= Q;
        if (ok) {
          const float psi = __fadd_rn(Ks[p], __ldg(&rec[p].a));
          if (psi <= best) {  // p falls within a lane: "<=" keeps the smaller p
            best = psi;
            bp = p;
          }
        }
        if (!__all_sync(kFull, ok)) break;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int op = __shfl_xor_sync(kFull, bp, o);
        if (ob < best || (ob == best && op < bp)) {
          best = ob;
          bp = op;
        }
      }
      if (best == CUDART_INF_F) bp = -1;
      K = __fadd_rn(best, __ldg(&rec[i - 1].ce));
      if (lane == 0) Ks[i] = K;
      if (pr) {
        const int k = (i - 1) & 31;
        if (lane == k) pv = bp;
        if (k == 31 || i == n) {
          if (lane <= k) pr[i - 1 - k + lane] = (PT)pv;
        }
      }
      __syncwarp();  // Ks[i] visible to every lane before the next position
    }
    const bool inf = K == CUDART_INF_F;
    inf_any |= inf;
    if (lane == 0) {
      const float c = inf ? CUDART_INF_F : (float)((double)K + Dn);
      if (BATCH) a.costs[out] = c;
      else a.cost[out] = c;
    }
  }
  const bool any_neg = __any_sync(kFull, neg);
  if (lane == 0) {
    if (any_neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
    if (inf_any) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
  }
}

template <typename PT, bool BATCH>
int launch_r(const RescueArgs& a, int wpb, size_t smem, int grid, cudaStream_t st) {
  auto k = split_rescue_kernel<PT, BATCH>;
  if (smem > 48u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  k<<<grid, wpb * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace

bool rescue_supported(int n_max) { return n_max >= 0 && rescue_per_warp(n_max) <= kRescueWarpMax; }

int launch_split_rescue(const RescueArgs& a, int64_t max_work, cudaStream_t st) {
  const size_t per = rescue_per_warp(a.n_max);
  const int wpb = (int)std::min<size_t>(kRescueMaxWarps, std::max<size_t>(1, kRescueCtaBudget / per));
  const size_t smem = (size_t)wpb * per;
  // a few CTAs per SM at most: the list is short unless the rings were far too small
  const int64_t want = (max_work + wpb - 1) / wpb;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 2 * (int64_t)num_sms()));
  if (a.batched) return launch_r<uint16_t, true>(a, wpb, smem, grid, st);
  if (a.pred && a.pred_dtype == SDP_PRED_U16) return launch_r<uint16_t, false>(a, wpb, smem, grid, st);
  return launch_r<int32_t, false>(a, wpb, smem, grid, st);
}

}  // namespace sdp

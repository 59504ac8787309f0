// split_plain.cu -- the plain per-scenario Split kernel (SDP_ALGO_PLAIN).
//
// One thread per scenario, demands read straight from HBM (no staging), and
// for every tour position i every capacity-feasible predecessor p is relaxed
// in turn: the masked min-plus column product of Eq. eqdpA,
//     J(i) = min_{p<i, load(s_{p+1..i}) <= Q} J(p) + W(p,i),
// in the K(i) = J(i) - D(i) form (see StepRec).  The K(p) history of each
// scenario lives in a global scratch array interleaved by thread slot so that
// a warp's accesses coalesce.  The same kernel, fed a list of scenario ids,
// recomputes the scenarios a deque kernel flagged where the warp kernel of
// split_rescue.cu does not apply: soft capacity, the adjoint's route counts,
// and rows too long for that kernel's shared memory.
#include <math_constants.h>

#include "sdp_internal.cuh"

namespace sdp {

// SOFT: every predecessor p is relaxed (the dense triangle of the penalised
// recursion), with beta per unit of route load above Q added to W(p,i).
template <typename PT, bool SOFT>
__global__ void __launch_bounds__(256) split_plain_kernel(SplitPlainArgs a) {
  const int64_t nslots = a.nslots;
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  const int n = a.n, Q = a.Q;
  const StepRec* __restrict__ rec = a.rec;
  float* Kb = a.kscratch + slot;
  const int64_t nwork = a.fb_list ? (int64_t)(*a.fb_count) : a.S;
  const double Dn = n > 0 ? *a.Dn : 0.0;
  bool neg = false, infeasible_any = false;
  for (int64_t w = slot; w < nwork; w += nslots) {
    const int64_t s = a.fb_list ? (int64_t)a.fb_list[w] : w;
    const int32_t* __restrict__ q = a.demands + s * n;
    PT* pr = a.pred ? (PT*)a.pred + s * n : nullptr;
    int32_t* ps = a.pscratch ? a.pscratch + slot : nullptr;
    float K = 0.f;
    Kb[0] = 0.f;
    for (int i = 1; i <= n; ++i) {
      const float ce = __ldg(&rec[i - 1].ce);
      float best = CUDART_INF_F;
      int bp = -1;
      int load = 0;
      for (int p = i - 1; p >= 0; --p) {
        int qp = __ldg(q + __ldg(&rec[p].col));  // customer at position p+1
        neg |= qp < 0;
        load += max(qp, 0);
        if (!SOFT && load > Q) break;
        float psi = __fadd_rn(Kb[(int64_t)p * nslots], __ldg(&rec[p].a));
        if (SOFT && load > Q) psi = __fadd_rn(psi, __fmul_rn(a.beta, (float)(load - Q)));
        if (psi <= best) {  // p descends: "<=" keeps the smallest p on ties
          best = psi;
          bp = p;
        }
      }
      if (best == CUDART_INF_F) bp = -1;
      K = __fadd_rn(best, ce);
      Kb[(int64_t)i * nslots] = K;
      if (pr) pr[i - 1] = (PT)bp;
      if (ps) ps[(int64_t)(i - 1) * nslots] = bp;
    }
    const bool inf = (K == CUDART_INF_F);
    infeasible_any |= inf;
    if (a.cost) a.cost[s] = inf ? CUDART_INF_F : (float)((double)K + Dn);
    if (a.hist && !inf) {
      // backtrack and count route starts / ends (adjoint)
      for (int i = n; i > 0;) {
        int p = pr ? (int)(long long)pr[i - 1] : ps[(int64_t)(i - 1) * nslots];
        if (sizeof(PT) == 2 && pr && p == 0xFFFF) break;
        if (p < 0 || p >= i) break;
        atomicAdd(&a.hist[p], 1ull);
        atomicAdd(&a.hist[n + i - 1], 1ull);
        i = p;
      }
      atomicAdd(&a.hist[2 * n], 1ull);
    }
  }
  if (neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  if (infeasible_any) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
}

int plain_grid(int device_sms) { return 2 * device_sms; }

void launch_split_plain(const SplitPlainArgs& a, int grid, cudaStream_t st) {
  const bool u16 = a.pred && a.pred_dtype == SDP_PRED_U16;
  if (a.soft) {
    if (u16) split_plain_kernel<uint16_t, true><<<grid, 256, 0, st>>>(a);
    else split_plain_kernel<int32_t, true><<<grid, 256, 0, st>>>(a);
  } else {
    if (u16) split_plain_kernel<uint16_t, false><<<grid, 256, 0, st>>>(a);
    else split_plain_kernel<int32_t, false><<<grid, 256, 0, st>>>(a);
  }
}

}  // namespace sdp

namespace sdp {

// Plain per-scenario Split for the batch entries the deque kernel flagged:
// entry g = b*S + s; thread slots reuse a K(p) scratch of n_max+1 floats.
__global__ void __launch_bounds__(256) batch_fallback_kernel(BatchFallbackArgs a) {
  const int64_t nslots = a.nslots;
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  float* Kb = a.kscratch + slot;
  const int64_t nwork = (int64_t)(*a.fb_count);
  for (int64_t w = slot; w < nwork; w += nslots) {
    const unsigned long long g = a.fb_list[w];
    const int b = (int)(g / (unsigned long long)a.S);
    const int64_t s = (int64_t)(g - (unsigned long long)b * a.S);
    const int n = a.n[b];
    const StepRec* __restrict__ rec = a.rec + a.rec_off[b];
    const int32_t* __restrict__ q = a.demands + a.dem_off[b] + s * n;
    float K = 0.f;
    Kb[0] = 0.f;
    for (int i = 1; i <= n; ++i) {
      float best = CUDART_INF_F;
      int load = 0;
      for (int p = i - 1; p >= 0; --p) {
        load += max(__ldg(q + __ldg(&rec[p].col)), 0);
        if (load > a.Q) break;
        const float psi = __fadd_rn(Kb[(int64_t)p * nslots], __ldg(&rec[p].a));
        best = psi <= best ? psi : best;
      }
      K = __fadd_rn(best, __ldg(&rec[i - 1].ce));
      Kb[(int64_t)i * nslots] = K;
    }
    a.costs[g] = K == CUDART_INF_F ? CUDART_INF_F : (float)((double)K + a.Dn[b]);
  }
}

void launch_batch_fallback(const BatchFallbackArgs& a, cudaStream_t st) {
  const int grid = (int)((a.nslots + 255) / 256);
  batch_fallback_kernel<<<grid, 256, 0, st>>>(a);
}

}  // namespace sdp

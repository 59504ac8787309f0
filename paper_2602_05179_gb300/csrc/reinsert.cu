// reinsert.cu -- backward Bellman DP of the order-up-to inventory reinsertion
// (Sec. 2 "Instantiation B", Eq. eqdp2; Algorithm "SolveBatchDP"), all T
// stages fused in one launch, then the backtrack from I0.
//
// Three kernels.  reinsert_kernel runs one scenario per warp (the two
// actions), reinsert_routes_kernel one scenario per warp with up to K route
// options, and reinsert_lane_kernel (below) one scenario per lane, for the
// two actions or up to 8 route options.  SDP_REINSERT_AUTO takes the lane
// kernel wherever it applies (U <= 255, T <= 4096, at least 4 warps' worth of
// its shared memory per SM; not with a table end cost and route options);
// SDP_REINSERT_WARP forces the warp kernels.
//
// Mapping of the warp kernels.  One warp per scenario; lane l owns the inventory states
// I = l + 32k, k < KC, so the consumption of the day is warp-uniform and the
// stage loop has no divergence.  With
//     G_{t+1}(j) = e(j) + C_{t+1}(max(0, j))      (e: end-of-day cost)
// both actions read one entry of G_{t+1}:
//     no delivery:  nd(I) = G_{t+1}(I - d_t)
//     delivery:     dv(I) = f_t + c (U - I) + G_{t+1}(U - d_t)   (I < U)
//     C_t(I) = min(nd, dv), decision = [dv < nd]  (ties: no delivery).
// G lives in a per-warp shared-memory double buffer indexed j + P for
// j in [-P, U] (P = 32; for j < -P the linear tail e(j) = p (-j) is evaluated
// directly).  Decisions are warp ballots, one 32-bit word per (t, k), kept in
// shared memory for the backtrack.
#include <climits>

#include <math_constants.h>

#include "sdp_internal.cuh"

namespace sdp {

constexpr int kPad = 32;

// Decision words of one stage: KC ballots, padded to 8 words so that lane 0
// stores them with two 16-byte shared stores.
__host__ __device__ constexpr int bits_stride(int kc) { return (kc + 7) & ~7; }

template <int KC, bool TABLE, bool UNIT>
__global__ void __launch_bounds__(512) reinsert_kernel(ReinsertArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int T = a.T, U = a.U;
  constexpr int GW = kPad + 32 * KC;
  constexpr int BS = bits_stride(KC);
  // CTA-shared per-day routing cost, then per warp: G double buffer,
  // decision words, consumption of the current scenario
  float* fixed_sm = reinterpret_cast<float*>(smem);
  const size_t fixed_bytes = ((size_t)T * 4 + 15) & ~(size_t)15;
  // 16-byte multiple: lane 0 stores decision words with 16-byte stores
  const size_t per_warp = (((size_t)2 * GW + (size_t)T * BS + (size_t)T) * 4 + 15) & ~(size_t)15;
  unsigned char* wb = smem + fixed_bytes + per_warp * warp;
  float* G0 = reinterpret_cast<float*>(wb);
  float* G1 = G0 + GW;
  uint32_t* bits = reinterpret_cast<uint32_t*>(G1 + GW);
  int32_t* dsm = reinterpret_cast<int32_t*>(bits + (size_t)T * BS);
  for (int t = threadIdx.x; t < T; t += blockDim.x) fixed_sm[t] = __ldg(a.fixed + t);
  __syncthreads();

  const float h = a.h, p = a.p, c = a.c;
  // per-slot constants: e(I) for I >= 0; the delivery's extra cost over the
  // stage base, c (U - I) for I < U and +inf at I >= U (q = 0 there)
  float eI[KC], cq[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int I = lane + 32 * k;
    const int Ic = min(I, U);
    eI[k] = TABLE ? __ldg(a.table + Ic) : __fmul_rn(h, (float)Ic);
    cq[k] = I < U ? (UNIT ? __fmul_rn(c, (float)(U - I)) : 0.f) : CUDART_INF_F;
  }
  const float e0 = TABLE ? __ldg(a.table) : 0.f;
  // e(j) for the negative region j = lane - P of the G buffer, without C
  const float eneg = TABLE ? e0 : __fmul_rn(p, (float)(kPad - lane));
  bool neg = false;

  for (int64_t s = (int64_t)blockIdx.x * nw + warp; s < a.S; s += (int64_t)gridDim.x * nw) {
    for (int t = lane; t < T; t += 32) {
      int d = a.cons[s * T + t];
      neg |= d < 0;
      dsm[t] = max(d, 0);
    }
    // stage T: C_T = 0, so G_T(j) = e(j)
    float* Gn = G0;
    float* Gc = G1;
#pragma unroll
    for (int k = 0; k < KC; ++k) Gn[kPad + lane + 32 * k] = eI[k];
    Gn[lane] = eneg;
    __syncwarp();
    float C[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) C[k] = 0.f;

    for (int t = T - 1; t >= 0; --t) {
      const int d = dsm[t];
      const float C0n = Gn[kPad] - e0;  // C_{t+1}(0); exact (e0 = 0 in linear mode)
      // G_{t+1}(j) for any j <= U
      auto gat = [&](int j) -> float {
        if (j >= -kPad) return Gn[j + kPad];
        return TABLE ? Gn[kPad] : __fadd_rn(C0n, __fmul_rn(p, (float)(-j)));
      };
      const float ft = fixed_sm[t];
      const float base = __fadd_rn(ft, gat(U - d));
      uint32_t w[KC];
      if (!UNIT && d <= kPad && ft >= 0.f) {
        // no unit cost and f_t >= 0: the delivery cost is `base` for every I,
        // and at I = U (where delivering means q = 0) base = f_t + nd >= nd,
        // so the comparison alone already keeps "no delivery" there
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const float nd = Gn[lane + 32 * k - d + kPad];
          const bool dec = base < nd;
          C[k] = dec ? base : nd;
          w[k] = __ballot_sync(0xffffffffu, dec);
        }
      } else if (d <= kPad) {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const float nd = Gn[lane + 32 * k - d + kPad];
          const float dv = __fadd_rn(base, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          w[k] = __ballot_sync(0xffffffffu, dec);
        }
      } else {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const float nd = gat(lane + 32 * k - d);
          const float dv = __fadd_rn(base, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          w[k] = __ballot_sync(0xffffffffu, dec);
        }
      }
      if (lane == 0) {
        uint32_t* row = bits + t * BS;
#pragma unroll
        for (int k0 = 0; k0 < BS; k0 += 4) {
          uint4 v;
          v.x = k0 + 0 < KC ? w[k0 + 0] : 0u;
          v.y = k0 + 1 < KC ? w[k0 + 1] : 0u;
          v.z = k0 + 2 < KC ? w[k0 + 2] : 0u;
          v.w = k0 + 3 < KC ? w[k0 + 3] : 0u;
          *reinterpret_cast<uint4*>(row + k0) = v;
        }
      }
      // G_t for the next (earlier) stage
      const float C0 = __shfl_sync(0xffffffffu, C[0], 0);
#pragma unroll
      for (int k = 0; k < KC; ++k) Gc[kPad + lane + 32 * k] = __fadd_rn(eI[k], C[k]);
      Gc[lane] = TABLE ? __fadd_rn(e0, C0) : __fadd_rn(C0, eneg);
      __syncwarp();
      float* tmp = Gn; Gn = Gc; Gc = tmp;
    }

    // value from I0, optional C_0 for every I
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k == (a.I0 >> 5)) v = C[k];
    v = __shfl_sync(0xffffffffu, v, a.I0 & 31);
    if (lane == 0) a.value[s] = v;
    if (a.value0) {
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int I = lane + 32 * k;
        if (I <= U) a.value0[s * (U + 1) + I] = C[k];
      }
    }
    // backtrack (every lane walks the same path; lane t%32 writes day t):
    // deliver -> max(0, U - d_t), else max(0, I - d_t)
    if (a.policy) {
      int I = a.I0;
      for (int t = 0; t < T; ++t) {
        const uint32_t wd = bits[t * BS + (I >> 5)];
        const int dec = (wd >> (I & 31)) & 1;
        if ((t & 31) == lane) a.policy[s * T + t] = (uint8_t)dec;
        I = max((dec ? U : I) - dsm[t], 0);
      }
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

// ----------------------------------------------------------- route options
// reinsert_routes_kernel: the warp-per-scenario recursion with K candidate
// routes per day (an entry of the transition matrix is a minimum over route
// options).  Route r on day t costs rcost[t][r] and carries the delivery
// q = U - I only if its residual capacity in this scenario, cap[s][t][r], is
// at least q.  Per state the delivery costs F(q) = min over those routes, so
//     dv(I) = F(U - I) + G_{t+1}(U - d_t) (+ c (U - I)),
// +inf when no route fits; the two-action recursion of reinsert_kernel is
// the case K = 1 with a roomy route (same FP32 operations, same bits).
// Decisions stay ballot bits (deliver or not); the backtrack recomputes the
// route that carried each delivery (the cheapest feasible one, the first on
// ties) and writes r + 1 to the policy.  Linear end-of-day costs only.
constexpr int kUnrolledRoutes = 8;

template <int KC, bool UNIT>
__global__ void __launch_bounds__(512) reinsert_routes_kernel(ReinsertArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int T = a.T, U = a.U, K = a.n_routes;
  constexpr int GW = kPad + 32 * KC;
  constexpr int BS = bits_stride(KC);
  // CTA-shared route costs [T*K]; per warp: G double buffer, decision words,
  // consumption and route capacities of the current scenario
  float* rcost_sm = reinterpret_cast<float*>(smem);
  const size_t rc_bytes = ((size_t)T * K * 4 + 15) & ~(size_t)15;
  const size_t per_warp =
      (((size_t)2 * GW + (size_t)T * BS + (size_t)T + (size_t)T * K) * 4 + 15) & ~(size_t)15;
  unsigned char* wb = smem + rc_bytes + per_warp * warp;
  float* G0 = reinterpret_cast<float*>(wb);
  float* G1 = G0 + GW;
  uint32_t* bits = reinterpret_cast<uint32_t*>(G1 + GW);
  int32_t* dsm = reinterpret_cast<int32_t*>(bits + (size_t)T * BS);
  int32_t* capsm = dsm + T;
  for (int i = threadIdx.x; i < T * K; i += blockDim.x) rcost_sm[i] = __ldg(a.route_cost + i);
  __syncthreads();

  const float h = a.h, p = a.p, c = a.c;
  float eI[KC], cq[KC];
  // route r carries the refill q = U - I of slot k iff its capacity is at
  // least qmin[k]: q itself, or INT_MAX where there is nothing to deliver
  // (q <= 0), so one compare per (route, slot) decides
  int qmin[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int I = lane + 32 * k;
    eI[k] = __fmul_rn(h, (float)min(I, U));
    cq[k] = UNIT ? __fmul_rn(c, (float)(U - I)) : 0.f;
    qmin[k] = U - I >= 1 ? U - I : INT_MAX;
  }
  const float eneg = __fmul_rn(p, (float)(kPad - lane));
  bool neg = false;

  for (int64_t s = (int64_t)blockIdx.x * nw + warp; s < a.S; s += (int64_t)gridDim.x * nw) {
    for (int t = lane; t < T; t += 32) {
      const int d = a.cons[s * T + t];
      neg |= d < 0;
      dsm[t] = max(d, 0);
    }
    const int32_t* capg = a.route_cap + s * (int64_t)T * K;
    for (int i = lane; i < T * K; i += 32) capsm[i] = __ldg(capg + i);
    float* Gn = G0;
    float* Gc = G1;
#pragma unroll
    for (int k = 0; k < KC; ++k) Gn[kPad + lane + 32 * k] = eI[k];
    Gn[lane] = eneg;
    __syncwarp();
    float C[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) C[k] = 0.f;

    for (int t = T - 1; t >= 0; --t) {
      const int d = dsm[t];
      const float C0n = Gn[kPad];  // C_{t+1}(0) (e(0) = 0)
      auto gat = [&](int j) -> float {
        if (j >= -kPad) return Gn[j + kPad];
        return __fadd_rn(C0n, __fmul_rn(p, (float)(-j)));
      };
      const float gUd = gat(U - d);
      // cheapest route that holds q (q >= 1; +inf when none does).  Up to
      // kUnrolledRoutes routes the loop is unrolled: a compare and a
      // predicated min per route and slot.
      float fb[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) fb[k] = CUDART_INF_F;
      const float* frow = rcost_sm + t * K;
      const int* crow = capsm + t * K;
      if (K <= kUnrolledRoutes) {
#pragma unroll
        for (int r = 0; r < kUnrolledRoutes; ++r) {
          if (r < K) {
            const float fr = frow[r];
            const int cr = crow[r];
#pragma unroll
            for (int k = 0; k < KC; ++k)
              if (cr >= qmin[k]) fb[k] = fminf(fb[k], fr);
          }
        }
      } else {
        for (int r = 0; r < K; ++r) {
          const float fr = frow[r];
          const int cr = crow[r];
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (cr >= qmin[k]) fb[k] = fminf(fb[k], fr);
        }
      }
      uint32_t w[KC];
      // one branch per day (d is warp-uniform): the direct shared loads when
      // every state's I - d stays inside the buffer's negative margin
      if (d <= kPad) {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const float nd = Gn[lane + 32 * k - d + kPad];
          float dv = __fadd_rn(fb[k], gUd);
          if (UNIT) dv = __fadd_rn(dv, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          w[k] = __ballot_sync(0xffffffffu, dec);
        }
      } else {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const float nd = gat(lane + 32 * k - d);
          float dv = __fadd_rn(fb[k], gUd);
          if (UNIT) dv = __fadd_rn(dv, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          w[k] = __ballot_sync(0xffffffffu, dec);
        }
      }
      if (lane == 0) {
        uint32_t* row = bits + t * BS;
#pragma unroll
        for (int k0 = 0; k0 < BS; k0 += 4) {
          uint4 v;
          v.x = k0 + 0 < KC ? w[k0 + 0] : 0u;
          v.y = k0 + 1 < KC ? w[k0 + 1] : 0u;
          v.z = k0 + 2 < KC ? w[k0 + 2] : 0u;
          v.w = k0 + 3 < KC ? w[k0 + 3] : 0u;
          *reinterpret_cast<uint4*>(row + k0) = v;
        }
      }
      const float C0 = __shfl_sync(0xffffffffu, C[0], 0);
#pragma unroll
      for (int k = 0; k < KC; ++k) Gc[kPad + lane + 32 * k] = __fadd_rn(eI[k], C[k]);
      Gc[lane] = __fadd_rn(C0, eneg);
      __syncwarp();
      float* tmp = Gn; Gn = Gc; Gc = tmp;
    }

    float v = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k == (a.I0 >> 5)) v = C[k];
    v = __shfl_sync(0xffffffffu, v, a.I0 & 31);
    if (lane == 0) a.value[s] = v;
    if (a.value0) {
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int I = lane + 32 * k;
        if (I <= U) a.value0[s * (U + 1) + I] = C[k];
      }
    }
    if (a.policy) {
      int I = a.I0;
      for (int t = 0; t < T; ++t) {
        const uint32_t wd = bits[t * BS + (I >> 5)];
        const bool dec = (wd >> (I & 31)) & 1u;
        int route = 0;
        if (dec) {  // the cheapest route that holds U - I, the first on ties
          const int q = U - I;
          float best = CUDART_INF_F;
          for (int r = 0; r < K; ++r) {
            const float fr = rcost_sm[t * K + r];
            if (capsm[t * K + r] >= q && fr < best) {
              best = fr;
              route = r + 1;
            }
          }
        }
        if ((t & 31) == lane) a.policy[s * T + t] = (uint8_t)route;
        I = max((dec ? U : I) - dsm[t], 0);
      }
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

// ------------------------------------------------------- one scenario per lane
// reinsert_lane_kernel: the same recursion with lane l of a warp running
// scenario s0 + l on its own (no ballots or shuffles).  Layout and order:
//  - G_{t+1} lives in shared memory laid out [row][lane] (every access of the
//    warp hits 32 banks whatever the lanes' consumptions), state I at row
//    I + P with P = 32 KC - (U + 1), so the top row is state U and rows
//    0 .. P-1 hold G_{t+1}(j) of the negative end-of-day inventories
//    j = -P .. -1 (C_{t+1}(0) plus the stockout cost), written at the start of
//    each day for the lanes' consumptions.
//  - G is overwritten in place by G_t: the rows are visited from the top down
//    in batches of 32, and a state's no-delivery read G_{t+1}(I - d_t) is at a
//    row <= its own, so it is never one the stage has already rewritten
//    (d_t >= 0).  A batch issues its 32 reads before its writes.
//  - One batch body serves every batch of a day (reads at immediate offsets)
//    while every lane's consumption is at most 32 (batch 0: at most P, with
//    the reads of the P rows below state 0 clamped to the buffer); a day with
//    more takes the general body, which evaluates the stockout tail.  Keeping
//    the bodies few keeps the code small: a fully unrolled stage of 224 states
//    overflowed the instruction cache.
//  - e(I) comes from a CTA-wide row-indexed table (four rows per broadcast
//    load), a table of zeros in the last stage, which stores C_0 rather than
//    G_0, so the value and the C_0 table are read straight from the buffer.
//  - Bit j of decision word k is row 32 k + j; the bits of the P rows below
//    state 0 are never read, and at I = U (where delivering is q = 0) the
//    decision is forced to "no delivery" -- with f_t >= 0 the comparison
//    already keeps it, and a day with f_t < 0 rewrites state U after its
//    batch.  When the policy is wanted the words of a day go to a per-warp
//    scratch slot in global memory, [tile parity][t][k][lane] (coalesced
//    stores), and the backtrack of a tile runs one day per stage day of the
//    next tile (the last tile's after its stage loop), so its dependent reads
//    of the words come back while the next tile computes.  The policy is
//    stored four days per 32-bit word where rows allow.
// Needs U < 256; up to eight warps (one CTA) per SM, 32 KC x 128 bytes of
// shared memory each.
constexpr int kLaneWarps = 8;
constexpr int kLaneMaxRoutes = 8;  // route options the lane kernel takes
template <int M>
struct IntTag {
  static constexpr int value = M;
};

// RK > 0: route options (at most RK of them, K = a.n_routes), linear end
// costs: the delivery from state I rides the cheapest route whose residual
// capacity in the lane's scenario holds U - I, F_t(I) = min over those of
// rcost[t][r] (the test is I >= U - cap[t][r], one compare per route against
// an immediate per row), dv(I) = F_t(I) + G_{t+1}(U - d_t) (+ c (U - I)): the
// FP32 operations of reinsert_routes_kernel, so its bits.  The backtrack
// recomputes the route of each delivery (the cheapest, the first on ties)
// and writes r + 1 to the policy.
template <int KC, bool TABLE, bool UNIT, int RK = 0>
__global__ void __launch_bounds__(kLaneWarps * 32, 1) reinsert_lane_kernel(ReinsertArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NI = 32 * KC;  // rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int T = a.T, U = a.U;
  const int P = NI - (U + 1);  // rows below state 0
  // shared: etab[NI] (e of each row), ztab[32] zeros, ptab[33] (p m for
  // m = 0..32), fixed[T], then per warp G[NI][32]
  float* etab = reinterpret_cast<float*>(smem);
  float* ztab = etab + NI;
  float* ptab = ztab + 32;
  float* fixed_sm = ptab + 36;
  float* rcost_sm = fixed_sm + T;  // RK > 0: route costs [T][K]
  const int K = RK > 0 ? a.n_routes : 0;
  const size_t off = (((size_t)NI + 32 + 36 + (size_t)T + (size_t)T * K) * 4 + 15) & ~(size_t)15;
  float* Gl = reinterpret_cast<float*>(smem + off) + (size_t)warp * NI * 32 + lane;
  const float h = a.h, p = a.p, c = a.c;
  for (int r = threadIdx.x; r < NI; r += blockDim.x) {
    const int I = r - P;
    etab[r] = I < 0 ? 0.f : (TABLE ? __ldg(a.table + I) : __fmul_rn(h, (float)I));
  }
  for (int m = threadIdx.x; m < 32; m += blockDim.x) ztab[m] = 0.f;
  for (int m = threadIdx.x; m < 36; m += blockDim.x) ptab[m] = __fmul_rn(p, (float)m);
  if (RK == 0)
    for (int t = threadIdx.x; t < T; t += blockDim.x) fixed_sm[t] = __ldg(a.fixed + t);
  for (int i = threadIdx.x; i < T * K; i += blockDim.x) rcost_sm[i] = __ldg(a.route_cost + i);
  __syncthreads();

  const int64_t slot = (int64_t)blockIdx.x * nwarps + warp;
  // decision word (parity, t, k) of this lane at dw[32 * ((parity * T + t) * KC + k)]
  uint32_t* dw = a.policy ? a.dscratch + slot * (int64_t)2 * T * KC * 32 + lane : nullptr;
  // policy rows of 4-byte multiples on an aligned base: four days per store
  const bool pol4 = (T & 3) == 0 && (reinterpret_cast<uintptr_t>(a.policy) & 3) == 0;
  const float e0 = TABLE ? etab[P] : 0.f;  // e(j) for j <= 0 in table mode
  bool neg = false;

  // ---- backtrack of a finished tile, one day at a time (see above)
  struct Backtrack {
    int I, t;        // path state at day t
    uint32_t w;      // decision word of day t at I (loaded a day ahead)
    uint32_t pw;     // policy bytes of the current 4-day group
    int d;           // consumption of day t
    const int32_t* crow;
    const int32_t* caps;  // RK > 0: the scenario's route capacities [T][K]
    uint8_t* prow;
    const uint32_t* words;
    bool live;
  } bt;
  bt.t = T;  // nothing to backtrack yet
  bt.I = 0; bt.w = 0u; bt.pw = 0u; bt.d = 0; bt.crow = a.cons; bt.caps = a.route_cap; bt.prow = nullptr;
  bt.words = nullptr; bt.live = false;
  auto bt_start = [&](const int32_t* crow, int64_t s, bool live, const uint32_t* words) {
    bt.I = a.I0;
    bt.t = 0;
    bt.pw = 0u;
    bt.crow = crow;
    if (RK > 0) bt.caps = a.route_cap + s * (int64_t)T * K;
    bt.prow = a.policy + s * T;
    bt.words = words;
    bt.live = live;
    bt.w = words[32 * ((bt.I + P) >> 5)];
    bt.d = live ? max(__ldg(crow), 0) : 0;
  };
  auto bt_day = [&]() {
    const int t = bt.t;
    const int dec = (int)((bt.w >> ((bt.I + P) & 31)) & 1u);
    int pv = RK > 0 ? 0 : dec;
    if (RK > 0 && dec) {  // the cheapest route that holds U - I, the first on ties
      const int q = U - bt.I;
      float best = CUDART_INF_F;
      for (int r = 0; r < K; ++r) {
        const float fr = rcost_sm[t * K + r];
        if (__ldg(bt.caps + t * K + r) >= q && fr < best) {
          best = fr;
          pv = r + 1;
        }
      }
    }
    if (pol4) {
      bt.pw |= (uint32_t)pv << (8 * (t & 3));
      if ((t & 3) == 3) {
        if (bt.live) *reinterpret_cast<uint32_t*>(bt.prow + (t - 3)) = bt.pw;
        bt.pw = 0u;
      }
    } else if (bt.live) {
      bt.prow[t] = (uint8_t)pv;
    }
    bt.I = max((dec ? U : bt.I) - bt.d, 0);
    bt.t = t + 1;
    if (t + 1 < T) {
      bt.w = bt.words[32 * ((t + 1) * KC + ((bt.I + P) >> 5))];
      bt.d = bt.live ? max(__ldg(bt.crow + t + 1), 0) : 0;
    }
  };

  const int64_t tiles = (a.S + 31) / 32;
  int parity = 0;
  for (int64_t tile = slot; tile < tiles; tile += (int64_t)gridDim.x * nwarps) {
    const int64_t s0 = tile * 32;
    const bool live = lane < a.S - s0;
    const int32_t* crow = a.cons + (s0 + (live ? lane : 0)) * T;
    const int32_t* caprow = RK > 0 ? a.route_cap + (s0 + (live ? lane : 0)) * (int64_t)T * K : nullptr;
    auto cons_at = [&](int t) -> int {
      const int d = __ldg(crow + t);
      neg |= live && d < 0;
      return live ? max(d, 0) : 0;
    };
    // stage T: C_T = 0, G_T = e (rows below state 0 are written per day)
#pragma unroll 8
    for (int r = 0; r < NI; ++r) Gl[32 * r] = etab[r];
    uint32_t* dwp = dw ? dw + 32 * (int64_t)parity * T * KC : nullptr;

    int d_next = cons_at(T - 1);
    int capn[RK > 0 ? RK : 1];  // the capacities of the next day processed
#pragma unroll
    for (int r = 0; r < (RK > 0 ? RK : 1); ++r)
      capn[r] = (RK > 0 && r < K) ? __ldg(caprow + (T - 1) * K + r) : 0;
    for (int t = T - 1; t >= 0; --t) {
      const int d = d_next;
      if (t > 0) d_next = cons_at(t - 1);  // one day ahead
      if (bt.t < T) bt_day();              // the previous tile's path
      const bool last = t == 0;
      const float G0 = Gl[32 * P];  // G_{t+1}(0) = e(0) + C_{t+1}(0)
      const float C0 = TABLE ? 0.f : G0;  // linear mode: e(0) = 0
      // G_{t+1}(j), j < 0: table e(0) + C(0) = G(0); linear C(0) + p (-j)
      auto gneg = [&](int mj) -> float { return TABLE ? G0 : __fadd_rn(C0, __fmul_rn(p, (float)mj)); };
      const float gUd = d <= U ? Gl[32 * (U + P - d)] : gneg(d - U);
      const float ft = RK > 0 ? 0.f : fixed_sm[t];
      const float base = __fadd_rn(ft, gUd);
      // route r holds the refill from state I iff I >= thr[r] = U - cap[t][r]
      int thr[RK > 0 ? RK : 1];
      float cr[RK > 0 ? RK : 1];
      if (RK > 0) {
#pragma unroll
        for (int r = 0; r < RK; ++r) {
          thr[r] = r < K ? U - capn[r] : 0x3FFFFFFF;
          cr[r] = r < K ? rcost_sm[t * K + r] : CUDART_INF_F;
          if (t > 0 && r < K) capn[r] = __ldg(caprow + (t - 1) * K + r);  // one day ahead
        }
      }
      const float* et = last ? ztab : etab;
      const int dmax = __reduce_max_sync(0xffffffffu, d);
      // rows below state 0 that this day reads at immediate offsets:
      // j = -1 .. -min(d, P)
      if (dmax <= 32) {
        const int mmax = min(dmax, P);
        for (int m = 1; m <= mmax; ++m)
          Gl[32 * (P - m)] = TABLE ? G0 : __fadd_rn(C0, ptab[m]);
      }
      // One batch of 32 rows r = 32k + j (state I = r - P): its 32 reads
      // first, then the updates.  MODE 0: reads at immediate offsets; 1:
      // reads clamped at row 0 (batch 0 with every d <= P); 2: general, the
      // stockout tail evaluated below state 0.
      auto batch = [&](int k, auto mode_tag) -> uint32_t {
        constexpr int MODE = decltype(mode_tag)::value;
        float v[32];
        if (MODE == 2) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int src = 32 * k + j - P - d;  // state read
            const float g = Gl[32 * (max(src, 0) + P)];
            v[j] = src >= 0 ? g : gneg(-src);
          }
        } else if (MODE == 1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = Gl[32 * max(32 * k + j - d, 0)];
        } else {
          const float* Gd = Gl - 32 * d;
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = Gd[32 * (32 * k + j)];
        }
        const float4* e4 = reinterpret_cast<const float4*>(et + (last ? 0 : 32 * k));
        // row 32 k + j is state I = 32 k + j - P: route r fits iff j >= tk[r]
        int tk[RK > 0 ? RK : 1];
#pragma unroll
        for (int r = 0; r < (RK > 0 ? RK : 1); ++r) tk[r] = RK > 0 ? thr[r] + P - 32 * k : 0;
        // four partial words: short dependency chains for the bit ORs
        uint32_t w4[4] = {0u, 0u, 0u, 0u};
        float* Gk = Gl + 32 * 32 * k;
#pragma unroll
        for (int q4 = 7; q4 >= 0; --q4) {
          const float4 ev = e4[q4];
          const float es[4] = {ev.x, ev.y, ev.z, ev.w};
#pragma unroll
          for (int u = 3; u >= 0; --u) {
            const int j = 4 * q4 + u;
            float dv = base;
            if (RK > 0) {
              float F = CUDART_INF_F;
#pragma unroll
              for (int r = 0; r < RK; ++r)
                if (j >= tk[r]) F = fminf(F, cr[r]);
              dv = __fadd_rn(F, gUd);
              if (UNIT) dv = __fadd_rn(dv, __fmul_rn(c, (float)(U + P - 32 * k) - (float)j));
            } else if (UNIT) {
              dv = __fadd_rn(base, __fmul_rn(c, (float)(U + P - 32 * k) - (float)j));
            }
            const bool dec = dv < v[j];
            const float C = dec ? dv : v[j];
            Gk[32 * j] = __fadd_rn(es[u], C);
            if (dec) w4[j >> 3] |= 1u << j;
          }
        }
        return (w4[0] | w4[1]) | (w4[2] | w4[3]);
      };
      // from the top down: a batch only reads rows at or below its own,
      // which later batches have not rewritten yet
      uint32_t* dwt = dwp ? dwp + 32 * t * KC : nullptr;
      uint32_t km = 0x7FFFFFFFu;  // the top row is state U: no delivery there
      if (dmax <= 32) {
#pragma unroll 1
        for (int k = KC - 1; k >= 1; --k) {
          const uint32_t w = batch(k, IntTag<0>{}) & km;
          if (dwt) dwt[32 * k] = w;
          km = ~0u;
        }
      } else {
#pragma unroll 1
        for (int k = KC - 1; k >= 1; --k) {
          const uint32_t w = batch(k, IntTag<2>{}) & km;
          if (dwt) dwt[32 * k] = w;
          km = ~0u;
        }
      }
      {
        const uint32_t w = (dmax <= P ? batch(0, IntTag<1>{}) : batch(0, IntTag<2>{})) & km;
        if (dwt) dwt[0] = w;
      }
      // at I = U delivering is q = 0: no delivery, C = G_{t+1}(U - d).  The
      // comparison chose it unless f_t < 0.
      if (RK > 0 || ft < 0.f) Gl[32 * (U + P)] = __fadd_rn(et[last ? 0 : U + P], gUd);
    }
    // the previous tile's path ends before this tile's starts
    while (bt.t < T) bt_day();
    // value, optional C_0 table (the buffer holds C_0 now)
    if (live) {
      a.value[s0 + lane] = Gl[32 * (a.I0 + P)];
      if (a.value0)
        for (int I = 0; I <= U; ++I) a.value0[(s0 + lane) * (U + 1) + I] = Gl[32 * (I + P)];
    }
    if (dwp) bt_start(crow, s0 + (live ? lane : 0), live, dwp);
    parity ^= 1;
  }
  while (bt.t < T) bt_day();
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

namespace {
template <int KC, bool TABLE, bool UNIT>
int launch_kc(const ReinsertArgs& a, cudaStream_t st) {
  auto k = reinsert_kernel<KC, TABLE, UNIT>;
  constexpr int GW = kPad + 32 * KC;
  const size_t per_warp =
      (((size_t)2 * GW + (size_t)a.T * bits_stride(KC) + (size_t)a.T) * 4 + 15) & ~(size_t)15;
  const size_t fixed_bytes = ((size_t)a.T * 4 + 15) & ~(size_t)15;
  int warps = 16;
  while (warps > 1 && fixed_bytes + per_warp * warps > 100 * 1024) warps >>= 1;
  const size_t smem = fixed_bytes + per_warp * warps;
  if (smem > 200 * 1024) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, warps * 32, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) occ = 1;
  const int64_t need = (a.S + warps - 1) / warps;
  const int grid = (int)imin64(need, (int64_t)occ * num_sms());
  if (grid > 0) k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <bool TABLE, bool UNIT>
int by_kc(const ReinsertArgs& a, cudaStream_t st) {
  const int kc = (a.U + 1 + 31) / 32;
  switch (kc) {
    case 1: return launch_kc<1, TABLE, UNIT>(a, st);
    case 2: return launch_kc<2, TABLE, UNIT>(a, st);
    case 3: return launch_kc<3, TABLE, UNIT>(a, st);
    case 4: return launch_kc<4, TABLE, UNIT>(a, st);
    case 5: return launch_kc<5, TABLE, UNIT>(a, st);
    case 6: return launch_kc<6, TABLE, UNIT>(a, st);
    case 7: return launch_kc<7, TABLE, UNIT>(a, st);
    case 8: return launch_kc<8, TABLE, UNIT>(a, st);
    default:
      if (kc <= 16) return launch_kc<16, TABLE, UNIT>(a, st);
      return launch_kc<32, TABLE, UNIT>(a, st);
  }
}

template <int KC, bool TABLE, bool UNIT, int RK = 0>
int launch_lane_kc(const ReinsertArgs& a, cudaStream_t st) {
  auto k = reinsert_lane_kernel<KC, TABLE, UNIT, RK>;
  const int nr = RK > 0 ? a.n_routes : 0;
  const int warps = reinsert_lane_warps(a.T, a.U, TABLE, nr);
  if (warps < 1) return (int)cudaErrorInvalidValue;
  const size_t smem = reinsert_lane_smem_for(a.T, a.U, TABLE, warps, nr);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t tiles = (a.S + 31) / 32;
  const int64_t need = (tiles + warps - 1) / warps;
  const int grid = (int)imin64(need, (int64_t)num_sms());
  if (grid > 0) k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <int KC, bool UNIT>
int launch_routes_kc(const ReinsertArgs& a, cudaStream_t st) {
  auto k = reinsert_routes_kernel<KC, UNIT>;
  constexpr int GW = kPad + 32 * KC;
  const size_t per_warp = (((size_t)2 * GW + (size_t)a.T * bits_stride(KC) + (size_t)a.T +
                            (size_t)a.T * a.n_routes) * 4 + 15) & ~(size_t)15;
  const size_t rc_bytes = ((size_t)a.T * a.n_routes * 4 + 15) & ~(size_t)15;
  int warps = 16;
  while (warps > 1 && rc_bytes + per_warp * warps > 100 * 1024) warps >>= 1;
  const size_t smem = rc_bytes + per_warp * warps;
  if (smem > 200 * 1024) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, warps * 32, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) occ = 1;
  const int64_t need = (a.S + warps - 1) / warps;
  const int grid = (int)imin64(need, (int64_t)occ * num_sms());
  if (grid > 0) k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <bool UNIT>
int routes_by_kc(const ReinsertArgs& a, cudaStream_t st) {
  switch ((a.U + 1 + 31) / 32) {
    case 1: return launch_routes_kc<1, UNIT>(a, st);
    case 2: return launch_routes_kc<2, UNIT>(a, st);
    case 3: return launch_routes_kc<3, UNIT>(a, st);
    case 4: return launch_routes_kc<4, UNIT>(a, st);
    case 5: return launch_routes_kc<5, UNIT>(a, st);
    case 6: return launch_routes_kc<6, UNIT>(a, st);
    case 7: return launch_routes_kc<7, UNIT>(a, st);
    default: return launch_routes_kc<8, UNIT>(a, st);
  }
}

template <bool TABLE, bool UNIT, int RK = 0>
int lane_by_kc(const ReinsertArgs& a, cudaStream_t st) {
  switch ((a.U + 1 + 31) / 32) {
    case 1: return launch_lane_kc<1, TABLE, UNIT, RK>(a, st);
    case 2: return launch_lane_kc<2, TABLE, UNIT, RK>(a, st);
    case 3: return launch_lane_kc<3, TABLE, UNIT, RK>(a, st);
    case 4: return launch_lane_kc<4, TABLE, UNIT, RK>(a, st);
    case 5: return launch_lane_kc<5, TABLE, UNIT, RK>(a, st);
    case 6: return launch_lane_kc<6, TABLE, UNIT, RK>(a, st);
    case 7: return launch_lane_kc<7, TABLE, UNIT, RK>(a, st);
    default: return launch_lane_kc<8, TABLE, UNIT, RK>(a, st);
  }
}
}  // namespace

size_t reinsert_lane_smem_for(int T, int U, bool /*table*/, int warps, int n_routes) {
  const int NI = 32 * ((U + 1 + 31) / 32);
  return ((((size_t)NI + 32 + 36 + (size_t)T + (size_t)T * n_routes) * 4 + 15) & ~(size_t)15) +
         (size_t)warps * NI * 32 * 4;
}

// Warps per CTA (one CTA per SM): as many as the shared memory holds, up to 8.
int reinsert_lane_warps(int T, int U, bool table, int n_routes) {
  int w = kLaneWarps;
  while (w > 0 && reinsert_lane_smem_for(T, U, table, w, n_routes) > 227 * 1024) --w;
  return w;
}

bool reinsert_lane_supported(int T, int U, int n_routes) {
  return U >= 0 && U < 256 && T >= 1 && T <= 4096 && n_routes >= 0 && n_routes <= kLaneMaxRoutes &&
         reinsert_lane_warps(T, U, true, n_routes) >= 4;
}

size_t reinsert_lane_smem(int T, int U, bool table) {
  return reinsert_lane_smem_for(T, U, table, reinsert_lane_warps(T, U, table, 0), 0);
}

size_t reinsert_lane_scratch_bytes(int T, int U) {
  const int KC = (U + 1 + 31) / 32;
  return (size_t)num_sms() * kLaneWarps * 2 * (size_t)T * KC * 32 * 4;
}

int launch_reinsert(const ReinsertArgs& a, cudaStream_t st) {
  if (a.S <= 0) return 0;
  const bool unit = a.c != 0.f;
  if (a.n_routes > 0) {  // route options: U <= 255, linear end costs (checked by the caller)
    if (a.U > 255 || a.table) return (int)cudaErrorInvalidValue;
    // AUTO takes the lane kernel where it applies (up to 8 routes)
    if ((a.algo == SDP_REINSERT_LANE || a.algo == SDP_REINSERT_AUTO) &&
        reinsert_lane_supported(a.T, a.U, a.n_routes)) {
      if (a.n_routes <= 4)
        return unit ? lane_by_kc<false, true, 4>(a, st) : lane_by_kc<false, false, 4>(a, st);
      return unit ? lane_by_kc<false, true, 8>(a, st) : lane_by_kc<false, false, 8>(a, st);
    }
    return unit ? routes_by_kc<true>(a, st) : routes_by_kc<false>(a, st);
  }
  // AUTO takes LANE where it applies: at T = 60, U = 200, S = 10^6 it runs in
  // 5.20 ms against 6.17 ms for WARP (a register-resident variant of WARP,
  // shifting the cost-to-go by warp shuffles, was measured at 6.59 ms: a
  // shuffle and a select cost what the shared load and store they replace
  // do, and WARP is issue-bound at 82%, not bound by shared memory)
  if ((a.algo == SDP_REINSERT_LANE || a.algo == SDP_REINSERT_AUTO) &&
      reinsert_lane_supported(a.T, a.U, 0)) {
    if (a.table) return unit ? lane_by_kc<true, true>(a, st) : lane_by_kc<true, false>(a, st);
    return unit ? lane_by_kc<false, true>(a, st) : lane_by_kc<false, false>(a, st);
  }
  if (a.table) return unit ? by_kc<true, true>(a, st) : by_kc<true, false>(a, st);
  return unit ? by_kc<false, true>(a, st) : by_kc<false, false>(a, st);
}

}  // namespace sdp

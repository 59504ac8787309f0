// reinsert.cu -- backward Bellman DP of the order-up-to inventory reinsertion
// (Sec. 2 "Instantiation B", Eq. eqdp2; Algorithm "SolveBatchDP"), all T
// stages fused in one launch, then the backtrack from I0.
//
// Mapping.  One warp per scenario; lane l owns the inventory states
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
#include <math_constants.h>

#include "sdp_internal.cuh"

namespace sdp {

constexpr int kPad = 32;

template <int KC, bool TABLE>
__global__ void __launch_bounds__(512) reinsert_kernel(ReinsertArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int T = a.T, U = a.U;
  const int GW = kPad + 32 * KC;
  const size_t per_warp = ((size_t)2 * GW + (size_t)T * KC + (size_t)T) * 4;
  unsigned char* wb = smem + per_warp * warp;
  float* G0 = reinterpret_cast<float*>(wb);
  float* G1 = G0 + GW;
  uint32_t* bits = reinterpret_cast<uint32_t*>(G1 + GW);
  int32_t* dsm = reinterpret_cast<int32_t*>(bits + (size_t)T * KC);

  const float h = a.h, p = a.p, c = a.c;
  // per-slot constants: e(I) for I >= 0, the delivery's unit part c (U - I)
  float eI[KC], cq[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int I = lane + 32 * k;
    const int Ic = min(I, U);
    eI[k] = TABLE ? __ldg(a.table + Ic) : __fmul_rn(h, (float)Ic);
    cq[k] = I < U ? __fmul_rn(c, (float)(U - I)) : CUDART_INF_F;
  }
  const float e0 = TABLE ? __ldg(a.table) : 0.f;
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
    Gn[lane] = TABLE ? e0 : __fmul_rn(p, (float)(kPad - lane));  // j = lane - P < 0
    __syncwarp();
    float C[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) C[k] = 0.f;

    for (int t = T - 1; t >= 0; --t) {
      const int d = dsm[t];
      const float C0n = Gn[kPad] - (TABLE ? e0 : 0.f);  // C_{t+1}(0) = G_{t+1}(0) - e(0)
      // G_{t+1}(j) for any j <= U
      auto gat = [&](int j) -> float {
        if (j >= -kPad) return Gn[j + kPad];
        return TABLE ? Gn[kPad] : __fadd_rn(C0n, __fmul_rn(p, (float)(-j)));
      };
      const float base = __fadd_rn(__ldg(a.fixed + t), gat(U - d));
      if (d <= kPad) {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const int I = lane + 32 * k;
          const float nd = Gn[I - d + kPad];
          const float dv = __fadd_rn(base, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          const uint32_t w = __ballot_sync(0xffffffffu, dec && I <= U);
          if (lane == 0) bits[t * KC + k] = w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const int I = lane + 32 * k;
          const float nd = gat(I - d);
          const float dv = __fadd_rn(base, cq[k]);
          const bool dec = dv < nd;
          C[k] = dec ? dv : nd;
          const uint32_t w = __ballot_sync(0xffffffffu, dec && I <= U);
          if (lane == 0) bits[t * KC + k] = w;
        }
      }
      // G_t for the next (earlier) stage
      const float C0 = __shfl_sync(0xffffffffu, C[0], 0);
#pragma unroll
      for (int k = 0; k < KC; ++k) Gc[kPad + lane + 32 * k] = __fadd_rn(eI[k], C[k]);
      Gc[lane] = TABLE ? __fadd_rn(e0, C0) : __fadd_rn(C0, __fmul_rn(p, (float)(kPad - lane)));
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
    // backtrack (every lane walks the same path; lane t%32 writes day t)
    if (a.policy) {
      int I = a.I0;
      for (int t = 0; t < T; ++t) {
        const uint32_t w = bits[t * KC + (I >> 5)];
        const int dec = (w >> (I & 31)) & 1;
        if ((t & 31) == lane) a.policy[s * T + t] = (uint8_t)dec;
        const int x = I + (dec ? U - I : 0) - dsm[t];
        I = max(x, 0);
      }
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

namespace {
template <int KC, bool TABLE>
int launch_kc(const ReinsertArgs& a, cudaStream_t st) {
  auto k = reinsert_kernel<KC, TABLE>;
  const int GW = kPad + 32 * KC;
  const size_t per_warp = ((size_t)2 * GW + (size_t)a.T * KC + (size_t)a.T) * 4;
  int warps = 16;
  while (warps > 1 && per_warp * warps > 100 * 1024) warps >>= 1;
  const size_t smem = per_warp * warps;
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

template <bool TABLE>
int by_kc(const ReinsertArgs& a, cudaStream_t st) {
  const int kc = (a.U + 1 + 31) / 32;
  switch (kc) {
    case 1: return launch_kc<1, TABLE>(a, st);
    case 2: return launch_kc<2, TABLE>(a, st);
    case 3: return launch_kc<3, TABLE>(a, st);
    case 4: return launch_kc<4, TABLE>(a, st);
    case 5: return launch_kc<5, TABLE>(a, st);
    case 6: return launch_kc<6, TABLE>(a, st);
    case 7: return launch_kc<7, TABLE>(a, st);
    case 8: return launch_kc<8, TABLE>(a, st);
    default:
      if (kc <= 16) return launch_kc<16, TABLE>(a, st);
      return launch_kc<32, TABLE>(a, st);
  }
}
}  // namespace

int launch_reinsert(const ReinsertArgs& a, cudaStream_t st) {
  if (a.S <= 0) return 0;
  return a.table ? by_kc<true>(a, st) : by_kc<false>(a, st);
}

}  // namespace sdp

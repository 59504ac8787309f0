// split_fleet.cu -- fleet-limited Split (at most K routes) for sm_103a.
//
// The extensive model of Appendix A bounds the vehicles used per scenario
// (constraint eq:fleet_size); its giant-tour example has "three vehicles
// available".  With hard capacity as in Eq. eqdpA and at most K routes, the
// recursion gains a route-count dimension:
//     J_k(i) = min over capacity-feasible p < i of J_{k-1}(p) + W(p,i),
//     J_0(0) = 0, J_0(i > 0) = J_k(0) = +inf, cost = min_{k <= K} J_k(n),
// ties to the smallest p at every (k, i), then to the fewest routes.  In the
// K-form of sdp_internal.cuh, layer k is the window minimum of
// psi_{k-1}(p) = K_{k-1}(p) + a_{p+1} -- the Split recursion fed by the layer
// below -- and every layer has the same capacity window.
//
// split_fleet_kernel: one warp per scenario, the layers across its lanes:
// lane l's slot j holds layer k = 32 j + l + 1 (two slots: K <= 64).  Every
// lane walks the same positions i = 1..n in lockstep, so the demand of s_i
// and the tour record are broadcast loads; layer k's input psi_{k-1}(i-1) =
// K_{k-1}(i-1) + a_i comes from the lane below (a shuffle; lane 0 of slot 0
// takes layer 0: K_0(0) = 0, else +inf), and each lane keeps its layer's
// window candidates in a monotone deque (entries (psi bits, L(p) << 16 | p),
// rings [slot][entry][lane] in shared memory): pop the back while its psi is
// larger (an equal one is older: smallest p), push p = i - 1 unless its state
// is unreachable (+inf), pop the front while the route p+1..i exceeds Q; an
// empty window reads +inf (a demand above Q at position i empties it, and
// the first such position makes every later J infinite).  With route output, i - p of every
// (i, k) goes to the warp's scratch row [i][k] and lane 0 walks the optimal
// split back.  A deque that outgrows its ring flags the scenario and
// split_fleet_rescue_kernel recomputes it, one warp per scenario and the same
// FP32 operations as split_fleet_plain_kernel (one thread per scenario, every
// feasible p of every layer: PLAIN, and the recomputation for n too long for
// the rescue's shared memory).  Rings of 16 entries, with 24 warps per CTA,
// overflow on some scenarios of the n = 500, K = 42 workload but run it in
// 5.4 ms of kernel where 32 entries and 16 warps took 9.0 ms; the one-thread
// recomputation of the overflowing scenarios alone took 39 ms.
#include <math_constants.h>

#include <algorithm>

#include "sdp_internal.cuh"

namespace sdp {

namespace {

constexpr int kFRing = 16;                          // deque entries per layer and lane
constexpr uint32_t kFRingBytes = kFRing * 256u;     // one layer's ring for 32 lanes
constexpr int kFMaxWarps = 24;                      // warps per CTA at most (as shared memory allows)
constexpr int kFAhead = 8;                          // demands loaded ahead

__device__ __forceinline__ float flds(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 flds2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ void fsts2(uint32_t a, uint32_t x, uint32_t y) {
  asm volatile("st.shared.v2.u32 [%0], {%1,%2};" ::"r"(a), "r"(x), "r"(y) : "memory");
}

// One layer's deque of one lane (checked form: emptiness tests, any demand).
struct FleetDeque {
  uint32_t rb;          // shared address of the lane's entry in ring slot 0
  uint32_t head, tail;  // byte offsets (multiples of 256), unwrapped
  uint32_t fent;        // front entry L(p) << 16 | p
  float fpsi, bpsi, K;  // front psi, back psi, K_k(i) of the last position
  bool full;
  __device__ __forceinline__ uint32_t at(uint32_t off) const {
    return rb + (off & ((kFRing - 1) << 8));
  }
  __device__ __forceinline__ void init(uint32_t ring, int lane) {
    rb = ring + 8u * (uint32_t)lane;
    head = tail = 0u;
    fent = 0u;
    fpsi = CUDART_INF_F;
    bpsi = -CUDART_INF_F;
    K = CUDART_INF_F;
    full = false;
  }
  // push entry (psi, ent) of p = i-1, then drop expired fronts; Lc = L(i)<<16.
  // An unreachable state (psi = +inf) is not pushed: it could only be the
  // minimum of an empty window, which reads +inf anyway (pushed, such entries
  // would pile up behind each other over a long unreachable stretch).
  __device__ __forceinline__ void step(float psi, uint32_t ent, uint32_t Lc, uint32_t Qc,
                                       float ce) {
    if (psi != CUDART_INF_F) {
      while (bpsi > psi) {
        tail -= 256u;
        bpsi = tail == head ? -CUDART_INF_F : flds(at(tail - 256u));
      }
      if (tail == head) {
        fpsi = psi;
        fent = ent;
      }
      if (tail - head >= kFRingBytes) {  // full: flagged, restart at the new entry
        full = true;
        head = tail;
        fpsi = psi;
        fent = ent;
      }
      fsts2(at(tail), __float_as_uint(psi), ent);
      tail += 256u;
      bpsi = psi;
    }
    while (tail != head && ((Lc | 0xFFFFu) - fent) > Qc) {
      head += 256u;
      if (head != tail) {
        const uint2 e = flds2(at(head));
        fpsi = __uint_as_float(e.x);
        fent = e.y;
      }
    }
    if (tail == head) {  // nothing feasible in the window
      fpsi = CUDART_INF_F;
      bpsi = -CUDART_INF_F;
    }
    K = __fadd_rn(fpsi, ce);
  }
};

// KS: slots per lane (layers = 32 KS >= K); ROUTES: keep i - p of every
// (i, k) in the warp's scratch for the backtrack.
template <int KS, bool ROUTES>
__global__ void __launch_bounds__(kFMaxWarps * 32) split_fleet_kernel(SplitFleetArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = a.n, Q = a.Q, K = a.K;
  // shared: (a_i, ce_i) and columns of the tour | per warp: KS rings,
  // route boundaries
  float2* rec = reinterpret_cast<float2*>(smem);
  uint16_t* cols = reinterpret_cast<uint16_t*>(rec + n);
  const size_t head_bytes = (((size_t)n * 8 + (size_t)n * 2) + 255) & ~(size_t)255;
  const size_t per_warp = (size_t)KS * kFRingBytes + 256 * 4;
  unsigned char* wb = smem + head_bytes + per_warp * warp;
  const uint32_t rings = (uint32_t)__cvta_generic_to_shared(wb);
  int32_t* bounds = reinterpret_cast<int32_t*>(wb + (size_t)KS * kFRingBytes);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const StepRec r = a.rec[k];
    rec[k] = make_float2(r.a, r.ce);
    cols[k] = (uint16_t)r.col;
  }
  __syncthreads();
  const uint32_t Qh = (uint32_t)Q << 16, Qc = Qh | 0xFFFFu;
  const double Dn = *a.Dn;
  const int64_t wslot = (int64_t)blockIdx.x * nw + warp;
  // the warp's delta scratch: [i][k] uint16, 32 KS layers per position
  uint16_t* dsc = ROUTES ? a.dscratch + wslot * (int64_t)n * 32 * KS : nullptr;
  bool neg = false, any_fb = false, any_inf = false;
  for (int64_t s = wslot; s < a.S; s += (int64_t)gridDim.x * nw) {
    const int32_t* qrow = a.demands + s * n;
    FleetDeque dq[KS];
#pragma unroll
    for (int j = 0; j < KS; ++j) dq[j].init(rings + (uint32_t)j * kFRingBytes, lane);
    // demands of positions i .. i + kFAhead - 1 (broadcast loads, ahead)
    int qa[kFAhead];
#pragma unroll
    for (int u = 0; u < kFAhead; ++u) qa[u] = u < n ? __ldg(qrow + cols[u]) : 0;
    uint32_t Lc = 0u;  // L(i-1) << 16 (mod 2^32)
    uint32_t first_inf = (uint32_t)n + 1u;
    for (int i0 = 1; i0 <= n; i0 += kFAhead) {
#pragma unroll
      for (int u = 0; u < kFAhead; ++u) {
        const int i = i0 + u;
        if (i > n) break;
        const int q = qa[u];
        qa[u] = i + kFAhead <= n ? __ldg(qrow + cols[i + kFAhead - 1]) : 0;
        neg |= q < 0;
        const uint32_t qh = (uint32_t)min(max(q, 0), Q + 1) << 16;
        if (qh > Qh && first_inf > (uint32_t)n) first_inf = (uint32_t)i;
        const float2 r = rec[i - 1];
        const uint32_t ent = Lc | (uint32_t)(i - 1);
        const uint32_t Lnew = Lc + qh;
        // inputs from the layer below as it stood before this position
        float below[KS];
#pragma unroll
        for (int j = 0; j < KS; ++j) {
          const float up = __shfl_up_sync(0xffffffffu, dq[j].K, 1);
          const float wrap = j > 0 ? __shfl_sync(0xffffffffu, dq[j > 0 ? j - 1 : 0].K, 31)
                                   : (i == 1 ? 0.f : CUDART_INF_F);
          below[j] = lane > 0 ? up : wrap;
        }
#pragma unroll
        for (int j = 0; j < KS; ++j) {
          if (32 * j + lane < K) {
            dq[j].step(__fadd_rn(below[j], r.x), ent, Lnew, Qc, r.y);
            if (ROUTES)
              dsc[(int64_t)(i - 1) * 32 * KS + 32 * j + lane] =
                  (uint16_t)(i - (int)(dq[j].fent & 0xFFFFu));
          }
        }
        Lc = Lnew;
      }
    }
    // the best layer k <= K, fewest routes on ties
    float best = CUDART_INF_F;
    int bk = 0;
    bool full = false;
#pragma unroll
    for (int j = KS - 1; j >= 0; --j) {
      if (32 * j + lane < K) {
        full |= dq[j].full;
        if (dq[j].K <= best) {
          best = dq[j].K;
          bk = 32 * j + lane + 1;
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
      if (ob < best || (ob == best && ok != 0 && (bk == 0 || ok < bk))) {
        best = ob;
        bk = ok;
      }
    }
    full = __any_sync(0xffffffffu, full);
    const bool infeasible = first_inf <= (uint32_t)n || bk == 0 || best == CUDART_INF_F;
    if (full) {
      if (lane == 0) {
        const uint32_t f = atomicAdd(a.fb_count, 1u);
        a.fb_list[f] = (uint32_t)s;
      }
      any_fb = true;
      continue;
    }
    any_inf |= infeasible;
    if (lane == 0) {
      a.cost[s] = infeasible ? CUDART_INF_F : (float)((double)best + Dn);
      if (a.nroutes) a.nroutes[s] = infeasible ? 0 : bk;
    }
    if (ROUTES) {
      uint8_t* ro = a.route + s * n;
      if (infeasible) {
        for (int m = lane; m < n; m += 32) ro[m] = 0xFFu;
      } else {
        // route k (1-based) covers positions bounds[k-1]+1 .. bounds[k]
        __syncwarp();
        if (lane == 0) {
          int i = n, k = bk;
          bounds[k] = n;
          while (k > 0) {
            if (i > 0) i = max(0, i - (int)dsc[(int64_t)(i - 1) * 32 * KS + (k - 1)]);
            bounds[--k] = i;
          }
        }
        __syncwarp();
        for (int m = lane; m < n; m += 32) {
          int k = 0;
          while (bounds[k + 1] <= m) ++k;
          ro[m] = (uint8_t)k;
        }
        __syncwarp();
      }
    }
  }
  if (lane == 0) {
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

// Every feasible p of every layer, one thread per scenario (PLAIN for the
// fleet-limited Split, and the recomputation of flagged scenarios): layer k
// from layer k - 1 held in the thread's scratch rows, the same FP32
// operations and tie rules as split_fleet_kernel.
__global__ void __launch_bounds__(256) split_fleet_plain_kernel(SplitFleetArgs a) {
  const int n = a.n, Q = a.Q, K = a.K;
  const int64_t nslots = a.nslots;
  const int64_t count = a.fb_list ? (int64_t)*a.fb_count : a.S;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < nslots;
       slot += (int64_t)gridDim.x * blockDim.x) {
    float* Kp = a.kscratch + slot * 2 * (int64_t)(n + 1);
    float* Kc = Kp + (n + 1);
    uint16_t* P = a.pscratch ? a.pscratch + slot * (int64_t)K * n : nullptr;
    for (int64_t it = slot; it < count; it += nslots) {
      const int64_t s = a.fb_list ? (int64_t)a.fb_list[it] : it;
      const int32_t* q = a.demands + s * n;
      Kp[0] = 0.f;
      for (int i = 1; i <= n; ++i) Kp[i] = CUDART_INF_F;
      float best = CUDART_INF_F;
      int bk = 0;
      bool infeasible = false;
      for (int i = 1; i <= n && !infeasible; ++i) infeasible = q[a.rec[i - 1].col] > Q;
      for (int k = 1; k <= K && !infeasible; ++k) {
        Kc[0] = CUDART_INF_F;
        for (int i = 1; i <= n; ++i) {
          float bv = CUDART_INF_F;
          int bp = -1;
          int load = 0;
          for (int p = i - 1; p >= 0; --p) {
            load += max(__ldg(q + a.rec[p].col), 0);
            if (load > Q) break;
            const float psi = __fadd_rn(Kp[p], a.rec[p].a);
            if (psi <= bv) {  // p runs downwards: the smallest p on ties
              bv = psi;
              bp = p;
            }
          }
          Kc[i] = bp < 0 ? CUDART_INF_F : __fadd_rn(bv, a.rec[i - 1].ce);
          if (P) P[(int64_t)(k - 1) * n + (i - 1)] = (uint16_t)(bp < 0 ? 0 : i - bp);
        }
        if (Kc[n] < best) {  // the fewest routes on ties
          best = Kc[n];
          bk = k;
        }
        float* t = Kp;
        Kp = Kc;
        Kc = t;
      }
      infeasible = infeasible || bk == 0 || best == CUDART_INF_F;
      a.cost[s] = infeasible ? CUDART_INF_F : (float)((double)best + *a.Dn);
      if (a.nroutes) a.nroutes[s] = infeasible ? 0 : bk;
      if (a.route) {
        uint8_t* ro = a.route + s * n;
        if (infeasible) {
          for (int m = 0; m < n; ++m) ro[m] = 0xFFu;
        } else {
          int i = n, k = bk;
          while (k > 0 && i > 0) {
            const int p = max(0, i - (int)P[(int64_t)(k - 1) * n + (i - 1)]);
            for (int m = p; m < i; ++m) ro[m] = (uint8_t)(k - 1);
            i = p;
            --k;
          }
        }
      }
      if (infeasible) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    }
  }
}

// Recomputation of the flagged scenarios, one warp per scenario.  Layer k
// depends only on layer k - 1, so within a layer every position is
// independent: lane l takes positions i = 1 + l, 33 + l, ... and scans its
// window p = i - 1 down to pmin(i), the smallest p whose route p+1..i fits Q
// (the same for every layer: found once per scenario by a binary search of
// the prefix loads).  K_{k-1} and K_k sit in shared memory, and the tour's
// a_{p+1} and ce_i once per CTA; the FP32 operations, the order of p and the
// tie rules are split_fleet_plain_kernel's, so the results are its bits, and
// the route deltas go to the same per-slot scratch for the same backtrack.
constexpr int kFRescueWarps = 8;
// per warp: K_{k-1}, K_k, prefix loads L and window starts pmin, [n+1] each
__host__ __device__ inline size_t fleet_rescue_per_warp(int n) { return (size_t)4 * 4 * ((size_t)n + 1); }
__host__ __device__ inline size_t fleet_rescue_head(int n) { return ((size_t)8 * (size_t)n + 15) & ~(size_t)15; }

__global__ void __launch_bounds__(kFRescueWarps * 32) split_fleet_rescue_kernel(SplitFleetArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int n = a.n, Q = a.Q, K = a.K;
  float* as = reinterpret_cast<float*>(smem);  // a_{p+1} at [p], ce_i at [n + i - 1]
  float* ces = as + n;
  float* Kp = reinterpret_cast<float*>(smem + fleet_rescue_head(n) + (size_t)wib * fleet_rescue_per_warp(n));
  float* Kc = Kp + (n + 1);
  int32_t* L = reinterpret_cast<int32_t*>(Kc + (n + 1));
  int32_t* pmin = L + (n + 1);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    as[k] = a.rec[k].a;
    ces[k] = a.rec[k].ce;
  }
  __syncthreads();
  const int64_t slot = (int64_t)blockIdx.x * wpb + wib;  // < nslots (the launch sees to it)
  uint16_t* P = a.pscratch ? a.pscratch + slot * (int64_t)K * n : nullptr;
  const int64_t count = (int64_t)*a.fb_count;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  for (int64_t it = slot; it < count; it += nw) {
    const int64_t s = (int64_t)a.fb_list[it];
    const int32_t* q = a.demands + s * n;
    __syncwarp();  // the previous scenario's reads are done
    int carry = 0;
    bool over = false;
    if (lane == 0) L[0] = 0;
    for (int i0 = 1; i0 <= n; i0 += 32) {
      const int i = i0 + lane;
      int v = 0;
      if (i <= n) {
        const int raw = __ldg(q + __ldg(&a.rec[i - 1].col));
        over |= raw > Q;
        v = max(raw, 0);
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
      }
      if (i <= n) L[i] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    const bool infeasible0 = __any_sync(0xffffffffu, over);
    __syncwarp();
    // pmin(i): L is non-decreasing, so the feasible p < i form [pmin, i - 1]
    // (pmin = i: none; only with a demand above Q, which makes the scenario
    // infeasible anyway)
    for (int i = 1 + lane; i <= n; i += 32) {
      const int Li = L[i];
      int lo = 0, hi = i;  // smallest p in [0, i) with Li - L[p] <= Q, else i
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (Li - L[mid] <= Q) hi = mid; else lo = mid + 1;
      }
      pmin[i] = lo;
    }
    for (int i = lane; i <= n; i += 32) Kp[i] = i == 0 ? 0.f : CUDART_INF_F;
    __syncwarp();
    float* kp = Kp;
    float* kc = Kc;
    float best = CUDART_INF_F;
    int bk = 0;
    for (int k = 1; k <= K && !infeasible0; ++k) {
      if (lane == 0) kc[0] = CUDART_INF_F;
      for (int i = 1 + lane; i <= n; i += 32) {
        const int pm = pmin[i];
        float bv = CUDART_INF_F;
        int bp = -1;
#pragma unroll 4
        for (int p = i - 1; p >= pm; --p) {
          const float psi = __fadd_rn(kp[p], as[p]);
          if (psi <= bv) {  // p runs downwards: the smallest p on ties
            bv = psi;
            bp = p;
          }
        }
        kc[i] = bp < 0 ? CUDART_INF_F : __fadd_rn(bv, ces[i - 1]);
        if (P) P[(int64_t)(k - 1) * n + (i - 1)] = (uint16_t)(bp < 0 ? 0 : i - bp);
      }
      __syncwarp();  // layer k complete before it is read
      if (kc[n] < best) {  // the fewest routes on ties
        best = kc[n];
        bk = k;
      }
      float* t = kp;
      kp = kc;
      kc = t;
    }
    const bool infeasible = infeasible0 || bk == 0 || best == CUDART_INF_F;
    if (lane == 0) {
      a.cost[s] = infeasible ? CUDART_INF_F : (float)((double)best + *a.Dn);
      if (a.nroutes) a.nroutes[s] = infeasible ? 0 : bk;
      if (infeasible) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    }
    if (a.route) {
      __syncwarp();  // the route deltas of every lane, for lane 0's backtrack
      uint8_t* ro = a.route + s * n;
      if (infeasible) {
        for (int m = lane; m < n; m += 32) ro[m] = 0xFFu;
      } else if (lane == 0) {
        int i = n, k = bk;
        while (k > 0 && i > 0) {
          const int p = max(0, i - (int)P[(int64_t)(k - 1) * n + (i - 1)]);
          for (int m = p; m < i; ++m) ro[m] = (uint8_t)(k - 1);
          i = p;
          --k;
        }
      }
    }
  }
}

size_t fleet_head(int n) { return (((size_t)n * 8 + (size_t)n * 2) + 255) & ~(size_t)255; }
size_t fleet_per_warp(int ks) { return (size_t)ks * kFRingBytes + 256 * 4; }

template <int KS, bool ROUTES>
int launch_fleet_k(const SplitFleetArgs& a, int warps, int grid, cudaStream_t st) {
  auto k = split_fleet_kernel<KS, ROUTES>;
  const size_t smem = fleet_head(a.n) + fleet_per_warp(KS) * warps;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace

// One CTA per SM with as many warps as its shared memory holds (up to 16);
// fewer CTAs when there are fewer scenarios.
FleetConfig fleet_config(int n, int K, int64_t S) {
  const int ks = K <= 32 ? 1 : 2;
  const size_t budget = 226 * 1024;  // dynamic shared memory of one CTA per SM
  const size_t head = fleet_head(n);
  int warps = head >= budget ? 0 : (int)((budget - head) / fleet_per_warp(ks));
  warps = warps > kFMaxWarps ? kFMaxWarps : warps;
  FleetConfig c{};
  c.warps = warps;
  if (warps < 1) return c;
  const int64_t need = (S + warps - 1) / warps;
  c.grid = (int)imin64(need < 1 ? 1 : need, (int64_t)num_sms());
  return c;
}

size_t fleet_dscratch_elems(int n, int K, const FleetConfig& c) {
  const int ks = K <= 32 ? 1 : 2;
  return (size_t)c.grid * c.warps * (size_t)n * 32 * ks;
}

int launch_split_fleet(const SplitFleetArgs& a, const FleetConfig& c, cudaStream_t st) {
  if (c.warps < 1) return (int)cudaErrorInvalidValue;
  if (a.K <= 32)
    return a.route ? launch_fleet_k<1, true>(a, c.warps, c.grid, st)
                   : launch_fleet_k<1, false>(a, c.warps, c.grid, st);
  return a.route ? launch_fleet_k<2, true>(a, c.warps, c.grid, st)
                 : launch_fleet_k<2, false>(a, c.warps, c.grid, st);
}

bool fleet_rescue_supported(int n) { return fleet_rescue_head(n) + fleet_rescue_per_warp(n) <= 200u * 1024u; }

int launch_split_fleet_rescue(const SplitFleetArgs& a, cudaStream_t st) {
  const size_t per = fleet_rescue_per_warp(a.n);
  int wpb = (int)std::min<size_t>(kFRescueWarps, std::max<size_t>(1, (96u * 1024u) / per));
  if (wpb > a.nslots) wpb = (int)a.nslots;
  const size_t smem = fleet_rescue_head(a.n) + (size_t)wpb * per;
  // one scratch slot per warp: wpb * grid <= nslots
  const int grid = (int)std::max<int64_t>(1, a.nslots / wpb);
  auto k = split_fleet_rescue_kernel;
  if (smem > 48u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  k<<<grid, wpb * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}

int launch_split_fleet_plain(const SplitFleetArgs& a, cudaStream_t st) {
  const int grid = (int)((a.nslots + 255) / 256);
  split_fleet_plain_kernel<<<grid, 256, 0, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace sdp

// split_stream.cu -- Split with the demands streamed in tour order
// (SDP_ALGO_STREAM) for sm_103a.
//
// Why.  The DEQUE kernels stage a whole demand row (indexed by customer) on
// chip and look each customer up as the tour reaches it.  Here the gather by
// customer is done by producer warps, tile by tile, while DP warps of the same
// CTA run the recursion on tiles produced earlier:
//
//   producers (8 warps): TMA bulk copies (cp.async.bulk + mbarrier, two
//     64 KB stages) bring R contiguous int32 demand rows into shared memory;
//     the warps narrow them to uint8 (Q <= 254) or uint16, clamp to [0, Q+1],
//     permute them into tour order (position i holds the demand of customer
//     s_i) and write rows of `stride` bytes to a workspace array with
//     coalesced 32-bit stores.  A finished 32-scenario tile is published by a
//     shared counter (release / acquire); rows with a demand above Q are
//     flagged per tile.
//   DP warps (16): one lane per scenario, 32 scenarios per warp; each lane
//     reads its own tour-ordered row 16 bytes at a time, one block ahead,
//     straight into registers (the rows were just written, so they are still
//     in L2).
//
// Producers are bound by HBM and the DP by the issue of its dependent
// compare / pop chain, so the two overlap on each SM; a CTA only waits for
// its own producers (no cross-CTA waits).
//
// DP (Eq. eqdpA in the K-form of sdp_internal.cuh): K(i) = min over the
// capacity window of psi(p) + ce_i, psi(p) = K(p) + a_{p+1}, kept in a
// monotone deque per lane (Algorithm "2D Kernel for Splitting", hard-capacity
// form).  A ring entry is the pair (psi bits, L(p) << 16 | p) with the prefix
// load L taken mod 2^16: every entry in the deque at step i has
// L(i-1) - L(p) <= Q, and the demand added at step i is at most Q + 1, so the
// differences the front test takes are below 2Q + 2 <= 65536 and exact mod
// 2^16 (Q <= 32767).  With Lp = L(i) << 16 | 0xFFFF, the test "route
// p+1..i exceeds Q" is the single unsigned compare
// Lp - entry > (Q << 16 | 0xFFFF).  Ring addresses are kept wrapped: each
// warp's ring is aligned to its own size, so the next slot is one add and one
// LOP3.  Ties keep the older entry (smallest p), as in every other kernel
// here, so costs and predecessors are bit-identical to DEQUE and PLAIN.
#include <math_constants.h>

#include "async_copy.cuh"
#include "sdp_internal.cuh"

namespace sdp {

namespace {

constexpr int kDpWarps = 16;                  // DP warps per CTA
constexpr int kProdWarps = 8;                 // producer warps per CTA
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kDpWarps + kProdWarps) * 32;
constexpr uint32_t kStage = 64u * 1024u;      // bytes per producer stage (two)
constexpr int kRing = 16;                     // deque ring entries per lane
constexpr uint32_t kRingBytes = (uint32_t)kRing * 256u;  // 32 lanes x 8 B per entry

// Barrier of the producer warps only (named barrier 1), OR-reducing v.
__device__ __forceinline__ bool prod_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(kProdThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void prod_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kProdThreads) : "memory");
}
// ------------------------------------------------------------------ the DP
// Demand of the u-th position of a 16-byte block, shifted to bits 16..31
// (uint8: 16 positions per block; uint16: 8).
template <typename QT>
__device__ __forceinline__ uint32_t q_hi(const uint4& v, int u) {
  constexpr int PER = 4 / (int)sizeof(QT);
  const int w = u / PER, e = u % PER;
  const uint32_t x = w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
  if (sizeof(QT) == 1) return __byte_perm(x, 0u, 0x4044u | ((uint32_t)e << 8));  // byte e -> byte 2
  return e == 0 ? (x << 16) : (x & 0xFFFF0000u);
}

// One lane's deque and DP state.  Each lane pops on its own (no warp votes:
// a vote waits for the warp to reconverge, which was measured slower).
template <bool CHECK>
struct StreamDP {
  uint32_t base;       // ring base of the warp (aligned to kRingBytes)
  uint32_t haddr;      // front slot
  uint32_t taddr;      // next free slot
  uint32_t Lp;         // CHECK: L(i) << 16 | 0xFFFF; else L(i) << 16 + i (mod 2^32)
  uint32_t fent;       // front entry: L(p) << 16 | p
  uint32_t first_inf;  // CHECK: first position with a demand above Q
  float K, bpsi, fpsi;
  bool full;           // the ring filled up: the scenario is recomputed

  __device__ __forceinline__ uint32_t wrap(uint32_t addr) const {
    return (addr & (kRingBytes - 1u)) | base;
  }
  __device__ __forceinline__ void init(uint32_t warp_base, int lane, float a1, int n) {
    base = warp_base;
    haddr = taddr = warp_base + 8u * (uint32_t)lane;
    Lp = CHECK ? 0xFFFFu : 0u;
    fent = 0u;
    first_inf = (uint32_t)n + 1u;
    K = 0.f;
    bpsi = -CUDART_INF_F;
    fpsi = a1;  // psi(0) = K(0) + a_1, the entry pushed by the first step
    full = false;
  }
  // Position i with demand qh (<< 16) and record r = (a_i, ce_i).
  //  Without a demand above Q (CHECK false): the entry of p = i-1 is the
  // previous Lp, and "route p+1..i exceeds Q" is (Lp - ent) > Qc with
  // Qc = Q << 16 | 0xFFFF (mod 2^32: the entries tested differ in prefix load
  // by at most 2Q < 2^16, and i - p < 2^16); a psi below the front's (the
  // deque's minimum) pops every entry, so the deque restarts at the new entry
  // and the back-pop loop needs no emptiness test; the newest entry never
  // pops from the front.
  __device__ __forceinline__ void step(int i, uint32_t qh, float2 r, uint32_t Qc, uint32_t Qh,
                                       int n) {
    if (!CHECK) {
      const float psi = __fadd_rn(K, r.x);
      const uint32_t ent = Lp;
      Lp += qh + 1u;
      if (psi < fpsi) {
        taddr = haddr;
        fpsi = psi;
        fent = ent;
        bpsi = -CUDART_INF_F;
      }
      while (bpsi > psi) {
        taddr = wrap(taddr - 256u);
        bpsi = lds_f32(wrap(taddr - 256u));
      }
      sts_u2(taddr, __float_as_uint(psi), ent);
      taddr = wrap(taddr + 256u);
      bpsi = psi;
      // the ring filled up: flagged (recomputed), and the deque restarts at
      // the new entry so that the ring keeps describing it and both loops end
      if (taddr == haddr) {
        full = true;
        haddr = wrap(taddr - 256u);
        fpsi = psi;
        fent = ent;
      }
      while (Lp - fent > Qc) {
        haddr = wrap(haddr + 256u);
        const uint2 e = lds_u2(haddr);
        fpsi = __uint_as_float(e.x);
        fent = e.y;
      }
      K = __fadd_rn(fpsi, r.y);
      return;
    }
    const float psi = __fadd_rn(K, r.x);
    const uint32_t ent = Lp - 0xFFFFu + (uint32_t)(i - 1);
    // back pops: an empty deque has bpsi = -inf
    while (bpsi > psi) {
      taddr = wrap(taddr - 256u);
      bpsi = taddr == haddr ? -CUDART_INF_F : lds_f32(wrap(taddr - 256u));
    }
    if (taddr == haddr) {  // emptied: the new entry becomes the front
      fpsi = psi;
      fent = ent;
    }
    const uint32_t naddr = taddr;
    sts_u2(naddr, __float_as_uint(psi), ent);
    taddr = wrap(taddr + 256u);
    bpsi = psi;
    full |= taddr == haddr;
    Lp += qh;
    if (CHECK && qh > Qh && first_inf > (uint32_t)n) first_inf = (uint32_t)i;
    // Front pops.  Without a demand above Q the newest entry (route s_i
    // alone) never pops; the guard keeps it in every case.
    while ((Lp - fent) > Qc && haddr != naddr) {
      haddr = wrap(haddr + 256u);
      const uint2 e = lds_u2(haddr);
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
    K = __fadd_rn(fpsi, r.y);
  }
  __device__ __forceinline__ int pred(int i) const {
    if (CHECK && (uint32_t)i >= first_inf) return -1;
    return (int)(fent & 0xFFFFu);
  }
};

// Predecessor output of one lane: positions are stored PACK at a time
// (PACK = 4, 2 or 1 as the row alignment allows).
template <typename PT, int PACK>
struct PredOut {
  PT* row;  // this lane's row, or NULL
  int buf[PACK];
  __device__ __forceinline__ void put(int slot, int p) { buf[slot] = p; }
  __device__ __forceinline__ void flush(int i0) {  // positions i0 .. i0+PACK-1 (1-based)
    if (!row) return;
    PT* dst = row + (i0 - 1);
    if (PACK == 4) {
      if (sizeof(PT) == 2)
        *reinterpret_cast<uint2*>(dst) = make_uint2(__byte_perm(buf[0], buf[1], 0x5410),
                                                    __byte_perm(buf[2], buf[3], 0x5410));
      else
        *reinterpret_cast<int4*>(dst) = make_int4(buf[0], buf[1], buf[2], buf[3]);
    } else if (PACK == 2) {
      if (sizeof(PT) == 2)
        *reinterpret_cast<uint32_t*>(dst) = __byte_perm(buf[0], buf[1], 0x5410);
      else
        *reinterpret_cast<int2*>(dst) = make_int2(buf[0], buf[1]);
    } else {
      *dst = (PT)buf[0];
    }
  }
};

// Tour records (a_i, ce_i) of position k + 1: from shared memory (one tour
// per launch) or through the read-only path from the plan's records.
struct SmemRec {
  const float2* p;
  __device__ __forceinline__ float2 operator()(int k) const { return p[k]; }
};
struct GlobalRec {
  const StepRec* p;
  int last;  // n - 1 (the look-ahead past position n reads position n)
  __device__ __forceinline__ float2 operator()(int k) const {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p + min(k, last)));
    return make_float2(v.y, v.z);
  }
};

// One 32-scenario tile: lane l runs scenario s0 + l over positions 1..n.
template <typename QT, typename PT, int PACK, bool CHECK, bool PRED, typename REC>
__device__ __forceinline__ void stream_tile(int n, int Q, const unsigned char* qrow,
                                            uint32_t ring_base, const REC rec2, int lane,
                                            PT* prow, float* K_out, uint32_t* first_inf,
                                            bool* bad) {
  constexpr int E = 16 / (int)sizeof(QT);  // positions per 16-byte block
  const uint32_t Qh = (uint32_t)Q << 16;
  const uint32_t Qc = Qh | 0xFFFFu;
  StreamDP<CHECK> st;
  float2 r = rec2(0);  // record of the next position, loaded one step ahead
  st.init(ring_base, lane, r.x, n);
  PredOut<PT, PACK> po{PRED ? prow : nullptr, {}};
  const int nblk = n / E;
  const uint4* src = reinterpret_cast<const uint4*>(qrow);
  uint4 cur = ld_cg_v4(src);
  for (int b = 0; b < nblk; ++b) {
    const uint4 nxt = ld_cg_v4(src + b + 1);  // rows carry >= 16 bytes of slack
    const int i0 = b * E + 1;
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const float2 rn = rec2(i0 + u);
      st.step(i0 + u, q_hi<QT>(cur, u), r, Qc, Qh, n);
      r = rn;
      if (PRED) {
        po.put(u % PACK, st.pred(i0 + u));
        if (u % PACK == PACK - 1) po.flush(i0 + u - (PACK - 1));
      }
    }
    cur = nxt;
  }
  // ragged tail: fewer than E positions, scalar predecessor stores
  for (int i = nblk * E + 1; i <= n; ++i) {
    const int u = i - 1 - nblk * E;
    const int w = u / (4 / (int)sizeof(QT)), e = u % (4 / (int)sizeof(QT));
    const uint32_t x = w == 0 ? cur.x : (w == 1 ? cur.y : (w == 2 ? cur.z : cur.w));
    const uint32_t qh = sizeof(QT) == 1 ? ((x >> (8 * e)) & 0xFFu) << 16
                                        : ((x >> (16 * e)) & 0xFFFFu) << 16;
    const float2 rn = rec2(i);
    st.step(i, qh, r, Qc, Qh, n);
    r = rn;
    if (PRED && prow) prow[i - 1] = (PT)st.pred(i);
  }
  *K_out = st.K;
  *first_inf = st.first_inf;
  *bad = st.full;
}

// --------------------------------------------------------------- producers
// Narrow + permute `rows` staged int32 demand rows (sq, n per row, by
// customer) into tour-ordered words: word k4 of row r holds positions
// PER*k4 .. PER*k4 + PER-1 (zero past n), clamped to [0, Q+1]; out row r
// starts at out + r * pitch (in words).  Work items (row, word) are dealt
// round-robin to the producer threads, (r, k4) advanced without a division.
// flag(r) is called for a row with a demand above Q; mn_all tracks the
// minimum demand (negative demands are reported by the caller).
template <typename QT, typename FLAG>
__device__ __forceinline__ void narrow_rows(const int32_t* sq, int rows, int n, int Q,
                                            const uint16_t* cols, int w4, uint32_t* out,
                                            int64_t pitch, int ptid, int& mn_all, FLAG flag) {
  constexpr int PER = 4 / (int)sizeof(QT);  // demands per 32-bit output word
  const int dr = kProdThreads / w4, dk = kProdThreads % w4;
  int r = ptid / w4, k4 = ptid % w4;
  const int items = rows * w4;
  for (int idx = ptid; idx < items; idx += kProdThreads) {
    int col[PER];
    if (sizeof(QT) == 1) {  // the 4 columns of word k4 in one 8-byte load
      const uint2 c4 = *reinterpret_cast<const uint2*>(cols + 4 * k4);
      col[0] = (int)(c4.x & 0xFFFFu);
      col[1] = (int)(c4.x >> 16);
      col[2 % PER] = (int)(c4.y & 0xFFFFu);
      col[3 % PER] = (int)(c4.y >> 16);
    } else {
      const uint32_t c2 = *reinterpret_cast<const uint32_t*>(cols + 2 * k4);
      col[0] = (int)(c2 & 0xFFFFu);
      col[1 % PER] = (int)(c2 >> 16);
    }
    const int32_t* srow = sq + r * n;
    int v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) v[e] = k4 * PER + e < n ? srow[col[e]] : 0;
    int mx = v[0], mn = v[0];
#pragma unroll
    for (int e = 1; e < PER; ++e) {
      mx = max(mx, v[e]);
      mn = min(mn, v[e]);
    }
    mn_all = min(mn_all, mn);
    uint32_t word;
    if (mx > Q || mn < 0) {  // clamp to [0, Q+1]; flag the row if above Q
      if (mx > Q) flag(r);
      word = 0;
#pragma unroll
      for (int e = 0; e < PER; ++e)
        word |= (uint32_t)min(max(v[e], 0), Q + 1) << (e * 8 * (int)sizeof(QT));
    } else if (sizeof(QT) == 1) {
      word = __byte_perm(__byte_perm(v[0], v[1], 0x0040), __byte_perm(v[2 % PER], v[3 % PER], 0x0040),
                         0x5410);
    } else {
      word = __byte_perm(v[0], v[1 % PER], 0x5410);
    }
    out[(int64_t)r * pitch + k4] = word;
    r += dr;
    k4 += dk;
    if (k4 >= w4) {
      k4 -= w4;
      ++r;
    }
  }
}

// Chunks of R rows (R | 32, R * n * 4 <= kStage) walk this CTA's tiles in
// order through the two stages.
template <typename QT>
__device__ __forceinline__ void produce(const StreamArgs& a, int R, int64_t tb, int64_t te,
                                        int32_t* const stage_ptr[2], const uint16_t* cols,
                                        uint32_t bar0, uint32_t bar1, uint32_t* ready,
                                        uint32_t* abort_flag) {
  const int n = a.n, Q = a.Q;
  const int64_t S = a.S;
  const int ptid = (int)threadIdx.x - kDpWarps * 32;
  const int subs = 32 / R;  // chunks per tile
  const int64_t nchunks = (te - tb) * subs;
  // chunk g = sub-chunk g % subs of tile tb + g / subs; rows may run past S
  auto chunk_row0 = [&](int64_t g) -> int64_t { return (tb + g / subs) * 32 + (g % subs) * R; };
  auto chunk_rows = [&](int64_t g) -> int {
    const int64_t r0 = chunk_row0(g);
    return r0 >= S ? 0 : (int)imin64(R, S - r0);
  };
  auto issue = [&](int64_t g, int b) {
    const int rows = chunk_rows(g);
    const uint32_t bytes = ((uint32_t)rows * (uint32_t)n * 4u) & ~15u;
    const uint32_t bar = b ? bar1 : bar0;
    mbar_arrive_tx(bar, bytes);
    if (bytes) bulk_g2s(smem_u32(stage_ptr[b]), a.demands + chunk_row0(g) * n, bytes, bar);
  };
  if (ptid == 0) {
    if (nchunks > 0) issue(0, 0);
    if (nchunks > 1) issue(1, 1);
  }
  const int w4 = (int)(a.stride / 4);  // 32-bit words per output row
  int mn_all = 0;
  int64_t g = 0;
  for (; g < nchunks; ++g) {
    const int b = (int)(g & 1);
    const uint32_t parity = (uint32_t)(g >> 1) & 1u;
    const bool ok = mbar_wait(b ? bar1 : bar0, parity);
    const int rows = chunk_rows(g);
    int32_t* sq = stage_ptr[b];
    const int64_t row0 = chunk_row0(g);
    // the last few demands of a ragged last chunk (not a whole 16 bytes)
    // come from global memory
    const int elems = rows * n;
    const int bulk_elems = (int)((((uint32_t)elems * 4u) & ~15u) >> 2);
    if (ok && ptid < elems - bulk_elems)
      sq[bulk_elems + ptid] = __ldg(a.demands + row0 * n + bulk_elems + ptid);
    if (prod_sync_or(!ok)) break;  // the producers leave together
    uint32_t* out = reinterpret_cast<uint32_t*>(a.qt + row0 * a.stride);
    narrow_rows<QT>(sq, rows, n, Q, cols, w4, out, w4, ptid, mn_all, [&](int r) {
      const int64_t sidx = row0 + r;
      atomicOr(&a.tflags[sidx >> 5], 1u << (sidx & 31));
    });
    // publish a finished tile: every producer's rows, then the counter
    const bool tile_done = (g % subs) == subs - 1;
    if (tile_done) __threadfence_block();
    prod_sync();  // also: the stage is free again
    if (ptid == 0) {
      // (a.stall: fault injection for tests -- no tile is published, and the
      // DP warps' waits run out after a.wait_ns)
      if (tile_done && !a.stall) st_release_shared(ready, (uint32_t)(g / subs + 1));
      if (g + 2 < nchunks) {
        fence_proxy_async();
        issue(g + 2, b);
      }
    }
  }
  if (g < nchunks) {
    // a copy never completed: stop the DP warps, let the copies in flight
    // land (again with a time limit) before shared memory goes
    if (ptid == 0) {
      atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
      st_release_shared(abort_flag, 1u);
      mbar_wait((g & 1) ? bar1 : bar0, (uint32_t)(g >> 1) & 1u);
      if (g + 1 < nchunks) mbar_wait(((g + 1) & 1) ? bar1 : bar0, (uint32_t)((g + 1) >> 1) & 1u);
    }
    prod_sync();
  }
  if (mn_all < 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

// Bounded wait of a DP warp for `need` published tiles; false on abort or
// time-out.
__device__ __forceinline__ bool wait_ready(const uint32_t* ready, const uint32_t* abort_flag,
                                           uint32_t need, uint64_t limit_ns) {
  if (ld_acquire_shared(ready) >= need) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (ld_acquire_shared(ready) >= need) return true;
    if (ld_acquire_shared(abort_flag)) return false;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(128);
  }
}

// ------------------------------------------------------------------ kernel
// One CTA per SM; CTA c owns tiles [c*T/G, (c+1)*T/G).
template <typename QT, typename PT, int PACK, bool PRED>
__global__ void __launch_bounds__(kThreads, 1) split_stream_kernel(StreamArgs a, int R) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t ready, abort_flag;
  const int n = a.n;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // shared: two stages | rings (aligned to their size) | records | columns
  int32_t* const stage_ptr[2] = {reinterpret_cast<int32_t*>(smem),
                                 reinterpret_cast<int32_t*>(smem + kStage)};
  const uint32_t s0addr = smem_u32(smem);
  const uint32_t rings = (s0addr + 2 * kStage + kRingBytes - 1) & ~(kRingBytes - 1);
  const uint32_t rec_s = rings + kRingBytes * kDpWarps;
  float2* rec2 = reinterpret_cast<float2*>(smem + (rec_s - s0addr));
  // columns of every position of a padded row (zero past n: the producers
  // read them in groups of 4 but use only positions below n)
  uint16_t* cols = reinterpret_cast<uint16_t*>(rec2 + n + 16);
  const int row_pos = (int)(a.stride / (int64_t)sizeof(QT));
  for (int k = threadIdx.x; k < n + 16; k += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (k < n) {
      const StepRec r = a.rec[k];
      v = make_float2(r.a, r.ce);
    }
    rec2[k] = v;
  }
  for (int k = threadIdx.x; k < row_pos; k += blockDim.x) cols[k] = k < n ? a.cols[k] : 0;
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_fence_init();
    ready = 0u;
    abort_flag = 0u;
  }
  __syncthreads();

  const int64_t tiles = (a.S + 31) / 32;
  const int64_t tb = tiles * blockIdx.x / gridDim.x;
  const int64_t te = tiles * (blockIdx.x + 1) / gridDim.x;
  if (warp >= kDpWarps) {
    produce<QT>(a, R, tb, te, stage_ptr, cols, bar0, bar1, &ready, &abort_flag);
    return;
  }

  const double Dn = *a.Dn;
  const uint32_t ring_base = rings + kRingBytes * (uint32_t)warp;
  uint32_t any_inf = 0, any_fb = 0;
  bool timed_out = false;
  for (int64_t lt = warp; tb + lt < te; lt += kDpWarps) {
    if (!wait_ready(&ready, &abort_flag, (uint32_t)(lt + 1), a.wait_ns)) {
      timed_out = !ld_acquire_shared(&abort_flag);
      st_release_shared(&abort_flag, 1u);  // the other DP warps stop waiting too
      break;
    }
    const int64_t tile = tb + lt;
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    const bool live = lane < rows;
    const unsigned char* qrow = a.qt + (s0 + (live ? lane : 0)) * a.stride;
    PT* prow = (PRED && live) ? reinterpret_cast<PT*>(a.pred) + (s0 + lane) * (int64_t)n : nullptr;
    const uint32_t tf = *reinterpret_cast<volatile const uint32_t*>(&a.tflags[tile]);
    float K;
    uint32_t first_inf;
    bool bad;
    if (tf)
      stream_tile<QT, PT, PACK, true, PRED>(n, a.Q, qrow, ring_base, SmemRec{rec2}, lane, prow, &K,
                                            &first_inf, &bad);
    else
      stream_tile<QT, PT, PACK, false, PRED>(n, a.Q, qrow, ring_base, SmemRec{rec2}, lane, prow, &K,
                                             &first_inf, &bad);
    bad = bad && live;
    if (live) {
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else {
        a.cost[s0 + lane] = first_inf <= (uint32_t)n ? CUDART_INF_F : (float)((double)K + Dn);
      }
    }
    any_inf |= tf;
    any_fb |= __ballot_sync(0xffffffffu, bad);
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (timed_out) atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
  }
}

// ------------------------------------------------------------ batched plan
// split_batch_stream_kernel: the same producer / DP split over the items of a
// batched plan.  A group is up to 16 consecutive 32-scenario tiles of one tour;
// groups are numbered longest tour first and claimed from the plan's counter
// by each CTA's producers.  The CTA's items (in claim order li = 0, 1, ...)
// go through a ring of kSlots row slots in a workspace array (32 rows of
// stride_max bytes each); DP warp w takes items w, w + 16, ...  A producer
// reuses slot li % kSlots only after DP warp li % 16 has finished the item
// that held it (per-warp done counters); after the last group it publishes
// the CTA's item count, which releases the DP warps.
constexpr int kSlots = 32;

template <typename QT>
__global__ void __launch_bounds__(kThreads, 1) split_batch_stream_kernel(BatchStreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t ready, final_count, done[kDpWarps], abort_flag;
  __shared__ uint32_t meta_inf[kSlots];
  __shared__ int32_t meta_b[kSlots];
  __shared__ int64_t meta_s0[kSlots];
  __shared__ int64_t group_id;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int Q = a.Q;
  // shared: two stages | rings (aligned to their size) | columns of a padded row
  int32_t* const stage_ptr[2] = {reinterpret_cast<int32_t*>(smem),
                                 reinterpret_cast<int32_t*>(smem + kStage)};
  const uint32_t s0addr = smem_u32(smem);
  const uint32_t rings = (s0addr + 2 * kStage + kRingBytes - 1) & ~(kRingBytes - 1);
  uint16_t* cols = reinterpret_cast<uint16_t*>(smem + (rings + kRingBytes * kDpWarps - s0addr));
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_fence_init();
    ready = 0u;
    final_count = 0xFFFFFFFFu;
    abort_flag = 0u;
  }
  if (threadIdx.x < kDpWarps) done[threadIdx.x] = 0u;
  __syncthreads();
  unsigned char* qslots = a.qt + (int64_t)blockIdx.x * kSlots * 32 * a.stride_max;
  const int64_t tpt = (a.S + 31) / 32;                 // tiles per tour
  const int64_t gpt = (tpt + kDpWarps - 1) / kDpWarps;  // groups per tour
  const int64_t groups = gpt * a.B;

  if (warp >= kDpWarps) {
    // ------------------------------------------------------------- producers
    const int ptid = (int)threadIdx.x - kDpWarps * 32;
    int cur_b = -1, n = 0, R = 32, subs = 1, w4 = 0;
    uint32_t li = 0;    // items claimed by this CTA so far
    int64_t gk = 0;     // chunks issued through the stages so far
    int mn_all = 0;
    bool failed = false;
    while (!failed) {
      if (ptid == 0) group_id = (int64_t)atomicAdd(a.counter, 1ull);
      prod_sync();
      const int64_t gid = group_id;
      if (gid >= groups) break;
      const int b = a.order[gid / gpt];
      const int64_t t0 = (gid % gpt) * kDpWarps;
      const int m = (int)imin64(kDpWarps, tpt - t0);  // items in the group
      if (b != cur_b) {  // this tour's columns, row geometry and chunking
        prod_sync();     // every producer is done with the old columns
        cur_b = b;
        n = a.n[b];
        const int row_pos = (int)(stream_row_stride(n, Q) / (int64_t)sizeof(QT));
        w4 = (int)(stream_row_stride(n, Q) / 4);
        const StepRec* rec = a.rec + a.rec_off[b];
        for (int k = ptid; k < row_pos; k += kProdThreads) cols[k] = k < n ? (uint16_t)rec[k].col : 0;
        R = 32;
        while ((size_t)R * n * 4 > kStage) R >>= 1;
        subs = 32 / R;
        prod_sync();
      }
      const int32_t* dem = a.demands + a.dem_off[b];
      // the group's chunks: item j, sub-chunk q -> rows t0*32 + j*32 + q*R ...
      const int nch = m * subs;
      auto crow0 = [&](int c) -> int64_t { return (t0 + c / subs) * 32 + (int64_t)(c % subs) * R; };
      auto crows = [&](int c) -> int {
        const int64_t r0 = crow0(c);
        return r0 >= a.S ? 0 : (int)imin64(R, a.S - r0);
      };
      auto issue = [&](int c, int st) {
        const uint32_t bytes = ((uint32_t)crows(c) * (uint32_t)n * 4u) & ~15u;
        const uint32_t bar = st ? bar1 : bar0;
        mbar_arrive_tx(bar, bytes);
        if (bytes) bulk_g2s(smem_u32(stage_ptr[st]), dem + crow0(c) * n, bytes, bar);
      };
      for (int c = 0; c < nch; ++c) {
        const uint32_t item = li + (uint32_t)(c / subs);
        const uint32_t slot = item % kSlots;
        if (c % subs == 0) {
          // the slot's previous item (item - kSlots) must be finished
          if (item >= kSlots) {
            const uint32_t need = (item - kSlots) / kDpWarps + 1;
            bool ok = true;
            if (ld_acquire_shared(&done[item % kDpWarps]) < need) {
              const uint64_t tw = global_ns();
              while (ld_acquire_shared(&done[item % kDpWarps]) < need) {
                if (global_ns() - tw > kWaitLimitNs) { ok = false; break; }
                __nanosleep(256);
              }
            }
            if (prod_sync_or(!ok)) { failed = true; break; }
          }
          if (ptid == 0) {
            meta_inf[slot] = 0u;
            meta_b[slot] = b;
            meta_s0[slot] = (t0 + c / subs) * 32;
          }
        }
        // two chunks in flight: issue this one and the next at the group's
        // start, later ones as their stage frees up
        if (ptid == 0) {
          if (c == 0) {
            issue(0, (int)(gk & 1));
            if (nch > 1) issue(1, (int)((gk + 1) & 1));
          }
        }
        const int st = (int)(gk & 1);
        const bool ok = mbar_wait(st ? bar1 : bar0, (uint32_t)(gk >> 1) & 1u);
        const int rows = crows(c);
        int32_t* sq = stage_ptr[st];
        const int elems = rows * n;
        const int bulk_elems = (int)((((uint32_t)elems * 4u) & ~15u) >> 2);
        if (ok && ptid < elems - bulk_elems)
          sq[bulk_elems + ptid] = __ldg(dem + crow0(c) * n + bulk_elems + ptid);
        if (prod_sync_or(!ok)) { failed = true; break; }
        const int rbase = (c % subs) * R;  // first row of the chunk within the item
        uint32_t* out = reinterpret_cast<uint32_t*>(qslots + ((int64_t)slot * 32 + rbase) * a.stride_max);
        narrow_rows<QT>(sq, rows, n, Q, cols, w4, out, a.stride_max / 4, ptid, mn_all,
                        [&](int r) { atomicOr(&meta_inf[slot], 1u << (rbase + r)); });
        const bool item_done = (c % subs) == subs - 1;
        if (item_done) __threadfence_block();
        prod_sync();  // also: the stage is free again
        ++gk;
        if (ptid == 0) {
          if (item_done) st_release_shared(&ready, item + 1);
          if (c + 2 < nch) {
            fence_proxy_async();
            issue(c + 2, (int)(gk + 1) & 1);
          }
        }
      }
      li += (uint32_t)m;
    }
    if (failed) {
      if (ptid == 0) {
        atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
        st_release_shared(&abort_flag, 1u);
        // let copies still in flight land before shared memory goes
        mbar_wait((gk & 1) ? bar1 : bar0, (uint32_t)(gk >> 1) & 1u);
        mbar_wait(((gk + 1) & 1) ? bar1 : bar0, (uint32_t)((gk + 1) >> 1) & 1u);
      }
      prod_sync();
    } else if (ptid == 0) {
      st_release_shared(&final_count, li);
    }
    if (mn_all < 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
    return;
  }

  // ------------------------------------------------------------------ DP warps
  const uint32_t ring_base = rings + kRingBytes * (uint32_t)warp;
  uint32_t any_inf = 0, any_fb = 0;
  bool timed_out = false;
  for (uint32_t k = 0;; ++k) {
    const uint32_t li = (uint32_t)warp + k * kDpWarps;
    // wait until item li is published or the producers are done
    bool have = ld_acquire_shared(&ready) > li;
    if (!have) {
      const uint64_t tw = global_ns();
      while (true) {
        if (ld_acquire_shared(&ready) > li) { have = true; break; }
        if (ld_acquire_shared(&final_count) <= li) break;
        if (ld_acquire_shared(&abort_flag) || global_ns() - tw > kWaitLimitNs) {
          timed_out = !ld_acquire_shared(&abort_flag);
          break;
        }
        __nanosleep(128);
      }
    }
    if (!have) break;
    const uint32_t slot = li % kSlots;
    const int b = meta_b[slot];
    const int64_t s0 = meta_s0[slot];
    const uint32_t tf = meta_inf[slot];
    const int n = a.n[b];
    const int rows = (int)imin64(32, a.S - s0);
    const bool live = lane < rows;
    const unsigned char* qrow = qslots + ((int64_t)slot * 32 + (live ? lane : 0)) * a.stride_max;
    const GlobalRec rec{a.rec + a.rec_off[b], n - 1};
    float K;
    uint32_t first_inf;
    bool bad;
    if (tf)
      stream_tile<QT, int32_t, 1, true, false>(n, Q, qrow, ring_base, rec, lane, nullptr, &K,
                                               &first_inf, &bad);
    else
      stream_tile<QT, int32_t, 1, false, false>(n, Q, qrow, ring_base, rec, lane, nullptr, &K,
                                                &first_inf, &bad);
    bad = bad && live;
    if (live) {
      const int64_t g = (int64_t)b * a.S + s0 + lane;
      if (bad) {
        const uint32_t f = atomicAdd(a.fb_count, 1u);
        a.fb_list[f] = (unsigned long long)g;
      } else {
        a.costs[g] = first_inf <= (uint32_t)n ? CUDART_INF_F : (float)((double)K + a.Dn[b]);
      }
    }
    any_inf |= tf;
    any_fb |= __ballot_sync(0xffffffffu, bad);
    __syncwarp();
    if (lane == 0) st_release_shared(&done[warp], k + 1);
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (timed_out) atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
  }
}

size_t batch_kernel_smem(int64_t stride_max) {
  return 2 * (size_t)kStage + kRingBytes * (kDpWarps + 1) + (((size_t)stride_max * 2 + 15) & ~(size_t)15);
}

size_t kernel_smem(int n, int64_t stride) {
  return 2 * (size_t)kStage + kRingBytes * (kDpWarps + 1)  // stages, rings + alignment slack
         + ((size_t)n + 16) * sizeof(float2)                // (a, ce) records
         + (((size_t)stride * 2 + 15) & ~(size_t)15);       // columns of a padded row
}

template <typename QT, typename PT, int PACK, bool PRED>
int launch_k(const StreamArgs& a, int R, cudaStream_t st) {
  auto k = split_stream_kernel<QT, PT, PACK, PRED>;
  const size_t smem = kernel_smem(a.n, a.stride);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t tiles = (a.S + 31) / 32;
  const int64_t sms = a.ctas_per_sm > 0 ? (int64_t)a.ctas_per_sm * num_sms() : num_sms();
  const int grid = (int)(tiles < sms ? tiles : sms);
  k<<<grid, kThreads, smem, st>>>(a, R);
  return (int)cudaGetLastError();
}

template <typename QT, typename PT>
int launch_pack(const StreamArgs& a, int R, int pack, cudaStream_t st) {
  if (!a.pred) return launch_k<QT, PT, 1, false>(a, R, st);
  if (pack == 4) return launch_k<QT, PT, 4, true>(a, R, st);
  if (pack == 2) return launch_k<QT, PT, 2, true>(a, R, st);
  return launch_k<QT, PT, 1, true>(a, R, st);
}

template <typename QT>
int launch_pt(const StreamArgs& a, int R, int pack, cudaStream_t st) {
  if (a.pred && a.pred_dtype == SDP_PRED_U16) return launch_pack<QT, uint16_t>(a, R, pack, st);
  return launch_pack<QT, int32_t>(a, R, pack, st);
}

}  // namespace

bool stream_supported(int n, int Q) { return n >= 1 && n <= kStreamMaxN && Q >= 1 && Q <= 32767; }

size_t stream_qt_bytes(int n, int Q, int64_t S) {
  return (size_t)(S * stream_row_stride(n, Q)) + 64;
}

int64_t batch_stream_stride(int n_max, int Q) { return stream_row_stride(n_max, Q); }

size_t batch_stream_qt_bytes(int n_max, int Q) {
  return (size_t)num_sms() * kSlots * 32 * (size_t)stream_row_stride(n_max, Q) + 64;
}

bool batch_stream_supported(int n_max, int Q) { return stream_supported(n_max, Q); }

int launch_split_batch_stream(const BatchStreamArgs& a, cudaStream_t st) {
  const size_t smem = batch_kernel_smem(a.stride_max);
  auto k = a.Q <= 254 ? split_batch_stream_kernel<uint8_t> : split_batch_stream_kernel<uint16_t>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k<<<num_sms(), kThreads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

int launch_split_stream(const StreamArgs& a0, cudaStream_t st) {
  StreamArgs a = a0;
  if (a.wait_ns == 0) a.wait_ns = kWaitLimitNs;  // unset: the default limit
  int R = 32;
  while (R > 1 && (size_t)R * a.n * 4 > kStage) R >>= 1;
  if (R < 4) return (int)cudaErrorInvalidValue;
  const int64_t tiles = (a.S + 31) / 32;
  cudaError_t e = cudaMemsetAsync(a.tflags, 0, sizeof(uint32_t) * (size_t)tiles, st);
  if (e != cudaSuccess) return (int)e;
  int pack = 1;
  if (a.pred) {
    const size_t pb = a.pred_dtype == SDP_PRED_U16 ? 2 : 4;
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.pred);
    if ((a.n & 3) == 0 && base % (4 * pb) == 0) pack = 4;
    else if ((a.n & 1) == 0 && base % (2 * pb) == 0) pack = 2;
  }
  return a.Q <= 254 ? launch_pt<uint8_t>(a, R, pack, st) : launch_pt<uint16_t>(a, R, pack, st);
}

}  // namespace sdp

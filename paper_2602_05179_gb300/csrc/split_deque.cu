// split_deque.cu -- the tuned Split kernels (SDP_ALGO_DEQUE) for sm_103a.
//
// Mapping.  One warp owns a tile of 32 scenarios (one per lane) at a time and
// walks the tour positions i = 1..n in lockstep, so the per-position tour
// record is a warp-uniform broadcast load (from shared memory).  Warps are
// independent: no CTA barrier inside the tile loop, and the grid is
// persistent.
//
// DP.  With K(i) = J(i) - D(i) (see StepRec), Eq. eqdpA is a sliding-window
// minimum: K(i) = min_{p in [pmin(i), i-1]} psi(p) + ce_i, psi(p) = K(p) +
// a_{p+1}, where both ends of the window only move forward.  Each lane keeps
// the window's candidates in a monotone deque (the linear split of Algorithm
// "2D Kernel for Splitting", in the form of Vidal 2016 for hard capacity):
//   - push p = i-1 after popping from the back every entry with a larger psi
//     (an entry with equal psi is older, so it stays: smallest p wins ties);
//   - pop from the front every entry whose route p+1..i exceeds Q, read from
//     the 16-bit prefix load stored with the entry;
//   - the front is the argmin (kept in registers).
// The deque is a ring of RING entries per lane in shared memory, laid out
// [entry][lane] so every access is bank-conflict free.  A scenario whose
// deque outgrows the ring is flagged and recomputed by the plain kernel.
//
// Demand staging (two variants of the same DP).
//   Shared memory: the tile's rows are contiguous in HBM (row-major [S, n]);
//   the warp reads them with coalesced 16-byte loads and stores them clamped
//   to Q+1 as uint8 (Q <= 254) or uint16, with a row stride whose word count
//   is odd, so the 32 lanes reading one column of 32 rows hit 32 banks.
//   Tensor memory (TMEM, 256 KB per SM, beside shared memory): lane l of the
//   warp's TMEM quadrant holds scenario l's row packed 4 (uint8) or 2 (uint16)
//   demands per 32-bit column; the column of customer s_i is warp-uniform, so
//   one tcgen05.ld.32x32b per step (issued a step ahead) delivers all 32
//   demands.  Shared memory then holds only the deque rings, so 16 warps fit
//   per SM instead of 8.
// While a tile is processed, the warp's next tile is prefetched into L2 with
// one bulk prefetch (cp.async.bulk.prefetch.L2).
//
// Outputs.  Predecessors are staged per 16 positions in a small shared buffer
// and written as coalesced row segments.  The fused adjoint instead writes the
// predecessor distance i - pred(i) in place over the consumed demand byte and
// backtracks it on chip into shared-memory route start / end histograms.
#include <math_constants.h>

#include "sdp_internal.cuh"

namespace sdp {

namespace {

__device__ __forceinline__ int4 ld_stream_v4(const int4* p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ int ld_stream_s32(const int32_t* p) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ int ld_s32(const int32_t* p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Bulk prefetch of [p, p+bytes) into L2 (executed by the TMA engine; p and
// bytes must be multiples of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes)
               : "memory");
}

// Warm L2 with `bytes` bytes at p (16-byte aligned interior only).
__device__ __forceinline__ void prefetch_region(const void* p, int64_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pa = (a + 15) & ~(uintptr_t)15;
  int64_t rem = ((bytes - (int64_t)(pa - a)) / 16) * 16;
  for (int64_t o = 0; rem > 0; o += 1 << 20, rem -= 1 << 20)
    prefetch_l2_bulk(reinterpret_cast<const void*>(pa + o), (uint32_t)imin64(rem, 1 << 20));
}

// Generic 16-byte record load (shared memory when the records fit, else
// global memory).
__device__ __forceinline__ StepRec ld_rec_any(const StepRec* p) {
  const int4 v = *reinterpret_cast<const int4*>(p);
  StepRec r;
  r.col = (uint32_t)v.x;
  r.a = __int_as_float(v.y);
  r.ce = __int_as_float(v.z);
  r.pad = 0u;
  return r;
}

// Record load from shared memory through its 32-bit shared address (a
// short-scoreboard LDS.128 instead of a generic load).
__device__ __forceinline__ StepRec ld_rec_shared(uint32_t saddr) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(saddr));
  StepRec r;
  r.col = (uint32_t)v.x;
  r.a = __int_as_float(v.y);
  r.ce = __int_as_float(v.z);
  r.pad = 0u;
  return r;
}

__device__ __forceinline__ int4 ld_v4(const int32_t* p) {
  int4 v;
  asm volatile("ld.global.nc.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// ------------------------------------------------------------------- TMEM
// Thin wrappers over the tcgen05 instructions used here (all .sync.aligned:
// every lane of the warp executes them together with the same address).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(a), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
               ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
  uint32_t v;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
  return v;
}
// Waits for this thread's outstanding tcgen05.ld; v is tied to the wait so
// that no use of the loaded value is scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t& v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(v)::"memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c,
                                         uint32_t d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
               ::"r"(taddr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ demand sources
// Shared-memory row of one scenario.
template <typename QT>
struct SmemQ {
  QT* row;
  int pending;
  __device__ __forceinline__ void prefetch(uint32_t col) { pending = (int)row[col]; }
  __device__ __forceinline__ int take(uint32_t /*col*/) { return pending; }
};

// TMEM row: 32-bit column c / (4 / sizeof(QT)) of the warp's lane.
template <typename QT>
struct TmemQ {
  uint32_t taddr;  // lane field = warp quadrant, column = first word of the row
  uint32_t word;
  __device__ __forceinline__ void prefetch(uint32_t col) {
    __syncwarp();  // the deque loops diverge; tcgen05 ops need the whole warp
    word = tmem_ld1(taddr + (sizeof(QT) == 1 ? (col >> 2) : (col >> 1)));
  }
  __device__ __forceinline__ int take(uint32_t col) {
    __syncwarp();
    tmem_wait_ld(word);
    if (sizeof(QT) == 1) return (int)((word >> ((col & 3u) * 8u)) & 0xFFu);
    return (int)((word >> ((col & 1u) * 16u)) & 0xFFFFu);
  }
};

struct TileFlags {
  uint32_t inf_rows;  // rows with a demand above Q
  bool zero;          // some demand <= 0 in the tile (routes may exceed 255)
  bool neg;
};

template <typename QT>
__device__ __forceinline__ void put_q(QT* qb, int rs_elems, int r, int c, int v, int Q,
                                      uint32_t& inf_rows, bool& zero, bool& neg) {
  neg |= v < 0;
  zero |= v <= 0;
  if (v > Q) inf_rows |= 1u << r;
  v = min(max(v, 0), Q + 1);
  qb[r * rs_elems + c] = (QT)v;
}

}  // namespace

// Staged demand row stride (bytes) for n customers: a multiple of 4 whose
// word count is odd (bank-conflict-free column reads across 32 rows).
__host__ __device__ __forceinline__ int staged_row_stride(int n, int qbytes) {
  int rs = (n * qbytes + 3) & ~3;
  if (((rs >> 2) & 1) == 0) rs += 4;
  return rs;
}

// 32-bit TMEM columns per scenario row (rounded up to the 4-column stores).
__host__ __device__ __forceinline__ int tmem_row_words(int n, int qbytes) {
  return (((n * qbytes + 3) / 4) + 3) & ~3;
}

namespace {

constexpr int kStagePitch = 33;  // predecessor stage: [16 positions][33] elements

// Coalesced 16-byte loads of `rows` contiguous demand rows of n int32 each,
// clamped to [0, Q+1] and stored as narrow shared-memory rows.
template <typename QT>
__device__ __forceinline__ TileFlags ingest_tile(const int32_t* src, int rows, int n,
                                                 int rs_elems, int Q, QT* qb, int lane) {
  uint32_t inf_rows = 0;
  bool zero = false, neg = false;
  const int64_t count = (int64_t)rows * n;
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && n >= 4;
  if (vec_ok) {
    const float inv_n = 1.0f / (float)n;
    const int64_t nvec = count >> 2;
    const int4* src4 = reinterpret_cast<const int4*>(src);
    constexpr int U = 4;
    for (int64_t v0 = lane; v0 < nvec; v0 += 32 * U) {
      int4 x[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (v0 + 32 * u < nvec) x[u] = ld_stream_v4(src4 + v0 + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t v = v0 + 32 * u;
        if (v >= nvec) break;
        const int f = (int)(v * 4);
        // row = f / n via an FP32 reciprocal (f < 2^21: off by at most one)
        int r = __float2int_rz(__int2float_rn(f) * inv_n);
        int c = f - r * n;
        if (c < 0) { --r; c += n; } else if (c >= n) { ++r; c -= n; }
        const int vals[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          int rr = r, cc = c + k;
          if (cc >= n) { cc -= n; ++rr; }
          put_q<QT>(qb, rs_elems, rr, cc, vals[k], Q, inf_rows, zero, neg);
        }
      }
    }
    for (int64_t f = (nvec << 2) + lane; f < count; f += 32) {
      const int r = (int)(f / n), c = (int)(f - (int64_t)r * n);
      put_q<QT>(qb, rs_elems, r, c, ld_stream_s32(src + f), Q, inf_rows, zero, neg);
    }
  } else {
    for (int64_t f = lane; f < count; f += 32) {
      const int r = (int)(f / n), c = (int)(f - (int64_t)r * n);
      put_q<QT>(qb, rs_elems, r, c, ld_stream_s32(src + f), Q, inf_rows, zero, neg);
    }
  }
  TileFlags t;
  t.inf_rows = __reduce_or_sync(0xffffffffu, inf_rows);
  t.zero = __any_sync(0xffffffffu, zero);
  t.neg = __any_sync(0xffffffffu, neg);
  return t;
}

// Lane r loads its own row (scenario s0 + r) and packs it into TMEM words,
// 4 x 32-bit columns per tcgen05.st; padding columns and lanes >= rows hold
// zeros.  Rows that start on 16 bytes (n % 4 == 0) are read 4 demands per
// load, 8 loads in flight per lane.
template <typename QT>
__device__ __forceinline__ uint32_t pack_q(const int* v, int Q, bool& zero, bool& neg,
                                           bool& inf) {
  constexpr int PER = 4 / (int)sizeof(QT);
  uint32_t word = 0;
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    int x = v[e];
    neg |= x < 0;
    zero |= x <= 0;
    inf |= x > Q;
    x = min(max(x, 0), Q + 1);
    word |= (uint32_t)x << (e * 8 * (int)sizeof(QT));
  }
  return word;
}

template <typename QT>
__device__ __forceinline__ TileFlags ingest_tile_tmem(const int32_t* src, int rows, int n,
                                                      int Q, uint32_t taddr, int lane) {
  constexpr int PER = 4 / (int)sizeof(QT);  // demands per word
  const int words = tmem_row_words(n, (int)sizeof(QT));
  const int32_t* row = src + (int64_t)lane * n;
  const bool live = lane < rows;
  bool zero = false, neg = false, inf = false;
  const bool vec = ((n & 3) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  if (vec) {
    constexpr int WPI = 8;  // words per iteration
    constexpr int LOADS = WPI * PER / 4;
    for (int w0 = 0; w0 < words; w0 += WPI) {
      int4 x[LOADS];
#pragma unroll
      for (int k = 0; k < LOADS; ++k) {
        const int c = w0 * PER + 4 * k;
        x[k] = (live && c < n) ? ld_v4(row + c) : make_int4(0, 0, 0, 0);
      }
      const int* xv = reinterpret_cast<const int*>(x);
      uint32_t pk[WPI];
#pragma unroll
      for (int k = 0; k < WPI; ++k) pk[k] = pack_q<QT>(xv + k * PER, Q, zero, neg, inf);
      tmem_st4(taddr + w0, pk[0], pk[1], pk[2], pk[3]);
      if (w0 + 4 < words) tmem_st4(taddr + w0 + 4, pk[4], pk[5], pk[6], pk[7]);
    }
  } else {
    for (int w0 = 0; w0 < words; w0 += 4) {
      int v[4 * PER];
#pragma unroll
      for (int k = 0; k < 4 * PER; ++k) {
        const int c = w0 * PER + k;
        v[k] = (live && c < n) ? ld_s32(row + c) : 0;
      }
      uint32_t pk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pk[k] = pack_q<QT>(v + k * PER, Q, zero, neg, inf);
      tmem_st4(taddr + w0, pk[0], pk[1], pk[2], pk[3]);
    }
  }
  tmem_wait_st();
  TileFlags t;
  t.inf_rows = __ballot_sync(0xffffffffu, inf && live);
  t.zero = __any_sync(0xffffffffu, zero);
  t.neg = __any_sync(0xffffffffu, neg);
  return t;
}

// Output modes of the DP
constexpr int kOutNone = 0;    // cost only (batched plans)
constexpr int kOutStream = 1;  // predecessors streamed out every 16 positions
constexpr int kOutDelta = 2;   // i - pred(i) written in place over the consumed
                               // demand byte (on-chip backtrack of the adjoint)

// Where the next tile's demand rows are warmed into L2: late in the current
// tile's DP, so that the prefetched bytes are not evicted before use.
struct NextTile {
  const void* ptr;   // nullptr: nothing to prefetch
  int64_t bytes;
  int at;            // first 16-position batch at or after this position
};

// The DP of one scenario per lane (see the file comment).  Every lane of the
// warp runs it (lanes >= rows on stale data, outputs dropped) so that TMEM
// loads and the 16-position output batches stay warp-collective.
// CHECK: the tile holds a scenario with a demand above Q; first_inf records
// the first such position of this lane's scenario.
// REC_SHARED: rec points to shared memory (loaded as LDS.128).
template <typename QT, typename PT, int RING, int OUT, bool CHECK, bool REC_SHARED,
          typename SRC>
__device__ __forceinline__ float dp_row(SRC src, QT* row, int n, int Q, const StepRec* rec,
                                        float* ring_psi, uint32_t* ring_meta, int lane,
                                        PT* stage, PT* pred_tile, int rows, bool check_delta,
                                        NextTile nxt, uint32_t& first_inf, bool& bad) {
  int head = 0, tail = 0;  // deque = ring[head .. tail)
  int L = 0;               // prefix load of the current position
  float K = 0.f;
  float bpsi = 0.f;        // psi of the back entry
  float fpsi = 0.f;        // the front entry: psi, prefix load, index
  int fL = 0, fidx = 0;
  const uint32_t rec_s = REC_SHARED ? (uint32_t)__cvta_generic_to_shared(rec) : 0u;
  auto load_rec = [&](int k) -> StepRec {
    if (REC_SHARED) return ld_rec_shared(rec_s + 16u * (uint32_t)k);
    return ld_rec_any(rec + k);
  };
  StepRec rn = load_rec(0);
  src.prefetch(rn.col);
  for (int i0 = 1; i0 <= n; i0 += 16) {
    const int ie = min(n, i0 + 15);
    if (nxt.ptr && lane == 0 && i0 <= nxt.at && nxt.at < i0 + 16)
      prefetch_region(nxt.ptr, nxt.bytes);
    for (int i = i0; i <= ie; ++i) {
      const StepRec r = rn;
      const int q = src.take(r.col);
      if (i < n) {
        rn = load_rec(i);
        src.prefetch(rn.col);
      }
      // push p = i-1 after dropping every back entry with a larger psi (an
      // equal psi stays: it is older, so the smallest p wins ties).  The
      // first pop is straight-line code; more pops are rare and looped.
      const float psi = __fadd_rn(K, r.a);
      const bool pb = tail > head && bpsi > psi;
      if (pb) {
        --tail;
        bpsi = ring_psi[((tail - 1) & (RING - 1)) * 32 + lane];
      }
      if (__any_sync(0xffffffffu, pb && tail > head && bpsi > psi)) {
        while (tail > head && bpsi > psi) {
          --tail;
          if (tail > head) bpsi = ring_psi[((tail - 1) & (RING - 1)) * 32 + lane];
        }
      }
      const int slot = (tail & (RING - 1)) * 32 + lane;
      ring_psi[slot] = psi;
      ring_meta[slot] = ((uint32_t)L << 16) | (uint32_t)(i - 1);
      const bool alone = tail == head;
      ++tail;
      bpsi = psi;
      if (alone) { fpsi = psi; fL = L; fidx = i - 1; }
      bad |= (tail - head) > RING;
      // extend the window's right end to customer s_i
      L += q;
      if (CHECK && q > Q && first_inf > (uint32_t)n) first_inf = (uint32_t)i;
      // drop predecessors whose route s_{p+1..i} exceeds Q (first pop
      // straight-line, further pops looped)
      const bool pf = tail - head > 1 && L - fL > Q;
      if (pf) {
        ++head;
        const int h = (head & (RING - 1)) * 32 + lane;
        fpsi = ring_psi[h];
        const uint32_t m = ring_meta[h];
        fidx = (int)(m & 0xFFFFu);
        fL = L - (int)(((uint32_t)L - (m >> 16)) & 0xFFFFu);  // 16-bit prefix load, widened
      }
      if (__any_sync(0xffffffffu, pf && tail - head > 1 && L - fL > Q)) {
        while (tail - head > 1 && L - fL > Q) {
          ++head;
          const int h = (head & (RING - 1)) * 32 + lane;
          fpsi = ring_psi[h];
          const uint32_t m = ring_meta[h];
          fidx = (int)(m & 0xFFFFu);
          fL = L - (int)(((uint32_t)L - (m >> 16)) & 0xFFFFu);
        }
      }
      K = __fadd_rn(fpsi, r.ce);
      if (OUT == kOutStream) {
        int p = fidx;
        if (CHECK && (uint32_t)i >= first_inf) p = -1;
        stage[(i - i0) * kStagePitch + lane] = (PT)p;
      } else if (OUT == kOutDelta) {
        const uint32_t delta = (uint32_t)(i - fidx);
        if (check_delta && delta > (sizeof(QT) == 1 ? 255u : 65535u)) bad = true;
        row[r.col] = (QT)delta;
      }
    }
    if (OUT == kOutStream) {
      // rows x positions [i0, ie] of the staged batch -> coalesced row segments
      __syncwarp();
      const int cnt = ie - i0 + 1;
      const int u = lane & 15;
      PT* dst = pred_tile + (int64_t)(lane >> 4) * n + (i0 - 1) + u;
      const PT* s = stage + u * kStagePitch + (lane >> 4);
      const int64_t step2 = 2 * (int64_t)n;
      if (u < cnt) {
#pragma unroll 4
        for (int r2 = 0; r2 < rows - (lane >> 4); r2 += 2) {
          *dst = s[r2];
          dst += step2;
        }
      }
      __syncwarp();
    }
  }
  return K;
}

}  // namespace

// ------------------------------------------------------------------ kernels
// Single tour, shared-memory staging (all output modes, incl. the adjoint).
template <typename QT, typename PT, int RING, int OUT>
__global__ void __launch_bounds__(256, 1) split_deque_kernel(SplitDequeArgs a,
                                                             int row_stride,
                                                             int64_t tiles, int rec_in_smem) {
  constexpr bool HIST = OUT == kOutDelta;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, Q = a.Q;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int rs_elems = row_stride / (int)sizeof(QT);

  // ---- CTA-shared: tour records, and (adjoint) columns + histograms
  size_t off = 0;
  const StepRec* rec = a.rec;
  if (rec_in_smem) {
    StepRec* rs = reinterpret_cast<StepRec*>(smem);
    for (int k = threadIdx.x; k < n; k += blockDim.x) rs[k] = a.rec[k];
    rec = rs;
    off += (size_t)n * sizeof(StepRec);
  }
  uint16_t* cols_sm = nullptr;
  unsigned int* hist_sm = nullptr;
  if (HIST) {
    cols_sm = reinterpret_cast<uint16_t*>(smem + off);
    off += ((size_t)n * 2 + 15) & ~(size_t)15;
    hist_sm = reinterpret_cast<unsigned int*>(smem + off);
    off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
    for (int k = threadIdx.x; k < n; k += blockDim.x) cols_sm[k] = a.cols[k];
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x) hist_sm[k] = 0u;
  }
  const size_t stage_bytes =
      OUT == kOutStream ? (((size_t)16 * kStagePitch * sizeof(PT) + 15) & ~(size_t)15) : 0;
  const size_t per_warp = (size_t)32 * row_stride + (size_t)RING * 32 * 8 + stage_bytes;
  unsigned char* wbase = smem + off + per_warp * warp;
  QT* qb = reinterpret_cast<QT*>(wbase);
  float* ring_psi = reinterpret_cast<float*>(wbase + (size_t)32 * row_stride);
  uint32_t* ring_meta = reinterpret_cast<uint32_t*>(ring_psi + RING * 32);
  PT* stage = reinterpret_cast<PT*>(ring_meta + RING * 32);
  __syncthreads();

  const double Dn = *a.Dn;
  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;

  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  for (int64_t tile = (int64_t)blockIdx.x * nwarps + warp; tile < tiles;
       tile += wstride) {
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    const TileFlags tf = ingest_tile<QT>(a.demands + s0 * n, rows, n, rs_elems, Q, qb, lane);
    neg |= tf.neg;
    NextTile nxt{nullptr, 0, 0};
    if (tile + wstride < tiles) {
      const int64_t ns0 = (tile + wstride) * 32;
      nxt = NextTile{a.demands + ns0 * n, imin64(32, a.S - ns0) * n * 4, (3 * n) / 4};
    }
    __syncwarp();

    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    QT* row = qb + lane * rs_elems;
    PT* pred_tile = a.pred ? reinterpret_cast<PT*>(a.pred) + s0 * n : nullptr;
    const bool valid = lane < rows;
    SmemQ<QT> src{row, 0};
    float K;
    if (tf.inf_rows)
      K = dp_row<QT, PT, RING, OUT, true, false>(src, row, n, Q, rec, ring_psi, ring_meta, lane,
                                                stage, pred_tile, pred_tile ? rows : 0, tf.zero,
                                                nxt, first_inf, bad);
    else
      K = dp_row<QT, PT, RING, OUT, false, false>(src, row, n, Q, rec, ring_psi, ring_meta,
                                                 lane, stage, pred_tile, pred_tile ? rows : 0,
                                                 tf.zero, nxt, first_inf, bad);
    bad = bad && valid;
    if (valid) {
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else if (a.cost) {
        a.cost[s0 + lane] = first_inf <= (uint32_t)n ? CUDART_INF_F
                                                      : (float)((double)K + Dn);
      }
    }
    any_inf |= tf.inf_rows;
    any_fb |= __ballot_sync(0xffffffffu, bad);
    // -------- fused adjoint: backtrack on chip, count route starts / ends
    if (HIST && valid && !bad && first_inf > (uint32_t)n) {
      for (int i = n; i > 0;) {
        const int p = i - (int)row[cols_sm[i - 1]];
        atomicAdd(&hist_sm[p], 1u);
        atomicAdd(&hist_sm[n + i - 1], 1u);
        i = p;
      }
      atomicAdd(&hist_sm[2 * n], 1u);
    }
    __syncwarp();
  }

  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  }
  if (HIST) {
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x)
      if (hist_sm[k]) atomicAdd(&a.hist[k], (unsigned long long)hist_sm[k]);
  }
}

// Single tour, TMEM staging (cost + streamed predecessors).  One CTA per SM
// (the dynamic shared memory request guarantees it) allocates all 512 TMEM
// columns; warp w uses its quadrant's lanes (w % 4) and column block w / 4.
template <typename QT, typename PT, int RING, int OUT>
__global__ void __launch_bounds__(512, 1) split_tmem_kernel(SplitDequeArgs a, int64_t tiles,
                                                            int rec_in_smem, int cols_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  const int n = a.n, Q = a.Q;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;

  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  size_t off = 0;
  const StepRec* rec = a.rec;
  if (rec_in_smem) {
    StepRec* rs = reinterpret_cast<StepRec*>(smem);
    for (int k = threadIdx.x; k < n; k += blockDim.x) rs[k] = a.rec[k];
    rec = rs;
    off += (size_t)n * sizeof(StepRec);
  }
  const size_t stage_bytes =
      OUT == kOutStream ? (((size_t)16 * kStagePitch * sizeof(PT) + 15) & ~(size_t)15) : 0;
  const size_t per_warp = (size_t)RING * 32 * 8 + stage_bytes;
  unsigned char* wbase = smem + off + per_warp * warp;
  float* ring_psi = reinterpret_cast<float*>(wbase);
  uint32_t* ring_meta = reinterpret_cast<uint32_t*>(ring_psi + RING * 32);
  PT* stage = reinterpret_cast<PT*>(ring_meta + RING * 32);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) +
                         (uint32_t)((warp >> 2) * cols_per_warp);

  const double Dn = *a.Dn;
  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;
  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  for (int64_t tile = (int64_t)blockIdx.x * nwarps + warp; tile < tiles; tile += wstride) {
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    const TileFlags tf = ingest_tile_tmem<QT>(a.demands + s0 * n, rows, n, Q, taddr, lane);
    neg |= tf.neg;
    NextTile nxt{nullptr, 0, 0};
    if (tile + wstride < tiles) {
      const int64_t ns0 = (tile + wstride) * 32;
      nxt = NextTile{a.demands + ns0 * n, imin64(32, a.S - ns0) * n * 4, (3 * n) / 4};
    }
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    PT* pred_tile = a.pred ? reinterpret_cast<PT*>(a.pred) + s0 * n : nullptr;
    const bool valid = lane < rows;
    TmemQ<QT> src{taddr, 0u};
    float K;
    if (tf.inf_rows)
      K = dp_row<QT, PT, RING, OUT, true, true>(src, (QT*)nullptr, n, Q, rec, ring_psi,
                                               ring_meta, lane, stage, pred_tile,
                                               pred_tile ? rows : 0, false, nxt, first_inf, bad);
    else
      K = dp_row<QT, PT, RING, OUT, false, true>(src, (QT*)nullptr, n, Q, rec, ring_psi,
                                                ring_meta, lane, stage, pred_tile,
                                                pred_tile ? rows : 0, false, nxt, first_inf, bad);
    bad = bad && valid;
    if (valid) {
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else if (a.cost) {
        a.cost[s0 + lane] = first_inf <= (uint32_t)n ? CUDART_INF_F
                                                      : (float)((double)K + Dn);
      }
    }
    any_inf |= tf.inf_rows;
    any_fb |= __ballot_sync(0xffffffffu, bad);
    __syncwarp();
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, 512);
}

// Batched Split: a persistent grid pulls work items (tour, 32-scenario tile)
// from a global counter; items are ordered longest tour first, so the uneven
// tours finish together.  Each warp grabs its next item before working on the
// current one and warms L2 with that item's demand rows.
template <typename QT, int RING>
__global__ void __launch_bounds__(256, 1) split_batch_kernel(BatchKernelArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Q = a.Q;
  const int row_bytes_max = staged_row_stride(a.n_max, (int)sizeof(QT));
  const size_t per_warp = (size_t)32 * row_bytes_max + (size_t)RING * 32 * 8;
  unsigned char* wbase = smem + per_warp * warp;
  QT* qb = reinterpret_cast<QT*>(wbase);
  float* ring_psi = reinterpret_cast<float*>(wbase + (size_t)32 * row_bytes_max);
  uint32_t* ring_meta = reinterpret_cast<uint32_t*>(ring_psi + RING * 32);
  const int64_t tiles = (a.S + 31) / 32;
  const int64_t items = tiles * a.B;
  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;

  auto pop = [&]() -> int64_t {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(a.counter, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, k, 0);
  };
  int64_t item = pop();
  while (item < items) {
    const int b = a.order[item / tiles];
    const int64_t s0 = (item % tiles) * 32;
    const int n = a.n[b];
    const int rows = (int)imin64(32, a.S - s0);
    const int rs_elems = staged_row_stride(n, (int)sizeof(QT)) / (int)sizeof(QT);
    const TileFlags tf = ingest_tile<QT>(a.demands + a.dem_off[b] + s0 * n, rows, n, rs_elems,
                                         Q, qb, lane);
    neg |= tf.neg;
    const int64_t next = pop();
    NextTile nxt{nullptr, 0, 0};
    if (next < items) {
      const int nb = a.order[next / tiles];
      const int64_t ns0 = (next % tiles) * 32;
      const int nn = a.n[nb];
      nxt = NextTile{a.demands + a.dem_off[nb] + ns0 * nn, imin64(32, a.S - ns0) * nn * 4,
                     (3 * n) / 4};
    }
    __syncwarp();
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    QT* row = qb + lane * rs_elems;
    const StepRec* rec = a.rec + a.rec_off[b];
    SmemQ<QT> src{row, 0};
    float K;
    if (tf.inf_rows)
      K = dp_row<QT, int32_t, RING, kOutNone, true, false>(src, row, n, Q, rec, ring_psi,
                                                           ring_meta, lane, nullptr, nullptr, 0,
                                                           false, nxt, first_inf, bad);
    else
      K = dp_row<QT, int32_t, RING, kOutNone, false, false>(src, row, n, Q, rec, ring_psi,
                                                            ring_meta, lane, nullptr, nullptr, 0,
                                                            false, nxt, first_inf, bad);
    const bool valid = lane < rows;
    bad = bad && valid;
    if (valid) {
      const int64_t g = (int64_t)b * a.S + s0 + lane;
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (unsigned long long)g;
      } else {
        a.costs[g] = first_inf <= (uint32_t)n ? CUDART_INF_F
                                               : (float)((double)K + a.Dn[b]);
      }
    }
    any_inf |= tf.inf_rows;
    any_fb |= __ballot_sync(0xffffffffu, bad);
    __syncwarp();
    item = next;
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  }
}

// ------------------------------------------------------------------ host side
bool deque_supported(int n, int Q) { return n >= 1 && n <= 65534 && Q >= 1 && Q <= 32767; }

namespace {
int out_mode(bool hist, bool want_pred) {
  return hist ? kOutDelta : (want_pred ? kOutStream : kOutNone);
}
size_t stage_bytes_for(int pred_bytes) {
  return pred_bytes > 0 ? (((size_t)16 * kStagePitch * pred_bytes + 15) & ~(size_t)15) : 0;
}
constexpr int kTmemWarps = 16;         // 4 warps per TMEM lane quadrant
constexpr int kTmemColsPerWarp = 128;  // 512 columns / 4 warps per quadrant
constexpr size_t kOneCtaPerSmSmem = 120 * 1024;
}  // namespace

DequeConfig deque_config(int n, int Q, int warps, int ring, bool hist, int pred_bytes,
                         bool allow_tmem) {
  DequeConfig c;
  c.qbytes = Q <= 254 ? 1 : 2;
  c.ring = ring;
  c.rec_in_smem = n <= 4096;
  c.row_stride = staged_row_stride(n, c.qbytes);
  const size_t rec = c.rec_in_smem ? (size_t)n * sizeof(StepRec) : 0;
  const size_t stage = hist ? 0 : stage_bytes_for(pred_bytes);
  // TMEM staging when the row fits a warp's 128 columns and no in-place
  // deltas are needed.
  c.tmem = allow_tmem && !hist && tmem_row_words(n, c.qbytes) <= kTmemColsPerWarp;
  if (c.tmem) {
    c.warps = kTmemWarps;
    const size_t need = rec + (size_t)c.warps * ((size_t)ring * 32 * 8 + stage);
    c.smem = need > kOneCtaPerSmSmem ? need : kOneCtaPerSmSmem;
    return c;
  }
  c.warps = warps > 0 ? warps : 4;
  size_t off = rec;
  if (hist) {
    off += ((size_t)n * 2 + 15) & ~(size_t)15;
    off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
  }
  c.smem = off + (size_t)c.warps * ((size_t)32 * c.row_stride + (size_t)ring * 32 * 8 + stage);
  return c;
}

namespace {
template <typename QT, typename PT, int RING, int OUT>
int launch_t(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
             int* occ_out) {
  const int64_t tiles = (a.S + 31) / 32;
  if (OUT != kOutDelta && c.tmem) {
    auto k = split_tmem_kernel<QT, PT, RING, OUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem);
    if (e != cudaSuccess) return (int)e;
    if (occ_out) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_out, k, c.warps * 32, c.smem);
      if (*occ_out > 1) *occ_out = 1;  // one TMEM owner per SM
      return (int)e;
    }
    k<<<grid, c.warps * 32, c.smem, st>>>(a, tiles, c.rec_in_smem ? 1 : 0, kTmemColsPerWarp);
    return (int)cudaGetLastError();
  }
  auto k = split_deque_kernel<QT, PT, RING, OUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)c.smem);
  if (e != cudaSuccess) return (int)e;
  if (occ_out) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_out, k, c.warps * 32, c.smem);
    return (int)e;
  }
  k<<<grid, c.warps * 32, c.smem, st>>>(a, c.row_stride, tiles, c.rec_in_smem ? 1 : 0);
  return (int)cudaGetLastError();
}

template <typename QT, typename PT, int OUT>
int by_ring(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
            int* occ) {
  switch (c.ring) {
    case 8: return launch_t<QT, PT, 8, OUT>(a, c, grid, st, occ);
    case 32: return launch_t<QT, PT, 32, OUT>(a, c, grid, st, occ);
    default: return launch_t<QT, PT, 16, OUT>(a, c, grid, st, occ);
  }
}

template <typename QT>
int by_out(const SplitDequeArgs& a, const DequeConfig& c, int mode, int grid,
           cudaStream_t st, int* occ) {
  if (mode == kOutDelta) return by_ring<QT, int32_t, kOutDelta>(a, c, grid, st, occ);
  if (mode == kOutNone) return by_ring<QT, int32_t, kOutNone>(a, c, grid, st, occ);
  if (a.pred_dtype == SDP_PRED_U16) return by_ring<QT, uint16_t, kOutStream>(a, c, grid, st, occ);
  return by_ring<QT, int32_t, kOutStream>(a, c, grid, st, occ);
}

int dispatch(const SplitDequeArgs& a, const DequeConfig& c, int mode, int grid,
             cudaStream_t st, int* occ) {
  if (c.qbytes == 1) return by_out<uint8_t>(a, c, mode, grid, st, occ);
  return by_out<uint16_t>(a, c, mode, grid, st, occ);
}
}  // namespace

int launch_split_deque(const SplitDequeArgs& a, const DequeConfig& c, int grid,
                       cudaStream_t st) {
  return dispatch(a, c, out_mode(a.hist != nullptr, a.pred != nullptr), grid, st, nullptr);
}

size_t batch_smem(int n_max, int Q, int warps, int ring) {
  const int qbytes = Q <= 254 ? 1 : 2;
  return (size_t)warps * ((size_t)32 * staged_row_stride(n_max, qbytes) + (size_t)ring * 32 * 8);
}

namespace {
template <typename QT, int RING>
int batch_t(const BatchKernelArgs& a, int warps, int grid, cudaStream_t st, int* occ) {
  auto k = split_batch_kernel<QT, RING>;
  const size_t smem = batch_smem(a.n_max, a.Q, warps, RING);
  if (occ) {  // configuration query (never during a stream capture)
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, warps * 32, smem);
  }
  k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}
template <typename QT>
int batch_ring(const BatchKernelArgs& a, int warps, int ring, int grid, cudaStream_t st, int* occ) {
  switch (ring) {
    case 8: return batch_t<QT, 8>(a, warps, grid, st, occ);
    case 32: return batch_t<QT, 32>(a, warps, grid, st, occ);
    default: return batch_t<QT, 16>(a, warps, grid, st, occ);
  }
}
}  // namespace

int launch_split_batch(const BatchKernelArgs& a, int warps, int ring, int grid, cudaStream_t st,
                       int* occ_out) {
  if (a.Q <= 254) return batch_ring<uint8_t>(a, warps, ring, grid, st, occ_out);
  return batch_ring<uint16_t>(a, warps, ring, grid, st, occ_out);
}

int deque_max_ctas_per_sm(const DequeConfig& c, bool hist, int pred_dtype,
                          bool want_pred, int* out) {
  SplitDequeArgs a{};
  a.pred_dtype = pred_dtype;
  return dispatch(a, c, out_mode(hist, want_pred), 0, nullptr, out);
}

}  // namespace sdp

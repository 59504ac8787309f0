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
// deque outgrows the ring is flagged and recomputed: by one warp
// (split_rescue.cu) for hard capacity, by the plain kernel for soft capacity
// and the adjoint.
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
//   per SM instead of 8 -- or 17..24 with fewer columns each when that many
//   finish every tile in one round where 16 would need two.
// (A bulk L2 prefetch of the next tile was measured: it raised DRAM reads from
// 2.2 to 3.8 GB per launch at n = 500, S = 10^6 -- prefetched lines were
// evicted before use -- for 3% less time, so tiles are read on demand, with
// 16 loads in flight per lane in the tensor-memory ingest.)
//
// Outputs.  Each lane stores its own predecessors 4 positions per store when
// n % 4 == 0 and the rows are aligned; otherwise they are staged per 16
// positions in a small shared buffer and written as coalesced row segments.
// The fused adjoint keeps the predecessor distance i - pred(i) instead -- in
// place over the consumed demand byte with shared-memory staging, in a
// lane-interleaved global scratch with TMEM staging -- and backtracks it on
// chip into shared-memory route start / end histograms.
#include <math_constants.h>

#include "sdp_internal.cuh"
#include "tmem.cuh"

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

// Generic 16-byte record load (shared memory when the records fit, else
// global memory).
__device__ __forceinline__ StepRec ld_rec_any(const StepRec* p) {
  const int4 v = *reinterpret_cast<const int4*>(p);
  StepRec r;
  r.col = (uint32_t)v.x;
  r.a = __int_as_float(v.y);
  r.ce = __int_as_float(v.z);
  r.pad = (uint32_t)v.w;
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
  r.pad = (uint32_t)v.w;
  return r;
}

__device__ __forceinline__ int4 ld_v4(const int32_t* p) {
  int4 v;
  asm volatile("ld.global.nc.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}


// ------------------------------------------------------------ demand sources
// Shared-memory row of one scenario: demand of customer r.col.
template <typename QT>
struct SmemQ {
  QT* row;
  int pending;
  __device__ __forceinline__ void prefetch(const StepRec& r) { pending = (int)row[r.col]; }
  __device__ __forceinline__ int take(const StepRec& /*r*/) { return pending; }
};

// TMEM row of the warp's lane.  The TMEM kernels rewrite their shared copy of
// the records (tmem_rec): col = the 32-bit column holding customer s_i's
// demand, pad = the byte-permute selector that extracts it.
template <typename QT>
__device__ __forceinline__ StepRec tmem_rec(StepRec r) {
  const uint32_t c = r.col;
  if (sizeof(QT) == 1) {
    r.col = c >> 2;
    r.pad = 0x4440u | (c & 3u);  // byte c % 4, upper bytes from the zero operand
  } else {
    const uint32_t b = 2u * (c & 1u);
    r.col = c >> 1;
    r.pad = 0x4400u | ((b + 1u) << 4) | b;  // half c % 2
  }
  return r;
}

// As tmem_rec, with the selector putting the demand at bits 16..31.
template <typename QT>
__device__ __forceinline__ StepRec tmem_rec16(StepRec r) {
  const uint32_t c = r.col;
  if (sizeof(QT) == 1) {
    r.col = c >> 2;
    r.pad = 0x4044u | ((c & 3u) << 8);  // byte c % 4 -> byte 2
  } else {
    const uint32_t b = 2u * (c & 1u);
    r.col = c >> 1;
    r.pad = 0x0044u | (b << 8) | ((b + 1u) << 12);  // half c % 2 -> bytes 2, 3
  }
  return r;
}

// HI: the records carry tmem_rec16 selectors (demand at bits 16..31).
template <typename QT, bool HI = false>
struct TmemQ {
  uint32_t taddr;  // lane field = warp quadrant, column = first word of the row
  uint32_t word;
  // Issued with the warp converged: at the start of a row and right after take.
  __device__ __forceinline__ void prefetch(const StepRec& r) { word = tmem_ld1(taddr + r.col); }
  __device__ __forceinline__ int take(const StepRec& r) {
    __syncwarp();  // the deque loops diverge; tcgen05 ops need the whole warp
    tmem_wait_ld(word);
    const uint32_t v = __byte_perm(word, 0u, r.pad);
    return (int)(HI ? v >> 16 : v);
  }
};

struct TileFlags {
  uint32_t inf_rows;  // rows with a demand above Q
  bool zero;          // some demand <= 0 in the tile (routes may exceed 255)
  bool neg;
  bool small_loads;   // every row's total demand is below 2^16 (n * max < 2^16)
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

// Bytes of the TMEM kernels' column / selector array (TmemGroup) after the
// records: positions 1 .. n plus 3 x 8 look-ahead copies.
__host__ __device__ __forceinline__ size_t cs_bytes(int n) {
  return (((size_t)n + 24) * 4 + 15) & ~(size_t)15;
}

// 32-bit TMEM columns per scenario row (rounded up to the 4-column stores).
__host__ __device__ __forceinline__ int tmem_row_words(int n, int qbytes) {
  return (((n * qbytes + 3) / 4) + 3) & ~3;
}

namespace {

constexpr int kBatch = 16;       // positions per predecessor output batch (16 or 32)
// Dynamic shared memory that keeps a TMEM-owning kernel at one CTA per SM.
constexpr size_t kOneCtaPerSmSmem = 120 * 1024;

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
  t.small_loads = false;
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

// Low bytes (uint8 rows) or halves (uint16 rows) of PER int32 demands packed
// into one word, element e at bits [e * 8 * sizeof(QT), ...).
template <typename QT>
__device__ __forceinline__ uint32_t pack_raw(const int* v) {
  if (sizeof(QT) == 1)
    return __byte_perm(__byte_perm(v[0], v[1], 0x0040), __byte_perm(v[2], v[3], 0x0040), 0x5410);
  return __byte_perm(v[0], v[1], 0x5410);
}

// WPI: 32-bit words per lane per iteration (WPI * 4 / sizeof(QT) / 4 16-byte
// loads in flight per lane).
template <typename QT, int WPI = 16>
__device__ __forceinline__ TileFlags ingest_tile_tmem(const int32_t* src, int rows, int n,
                                                      int Q, uint32_t taddr, int lane) {
  constexpr int PER = 4 / (int)sizeof(QT);  // demands per word
  const int words = tmem_row_words(n, (int)sizeof(QT));
  const int32_t* row = src + (int64_t)lane * n;
  const bool live = lane < rows;
  bool zero = false, neg = false, inf = false;
  const bool vec = ((n & 3) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  if (vec) {
    // Fast pass: pack without clamping, tracking each row's minimum and
    // maximum; a tile with a demand outside [0, Q] is packed again below with
    // the clamp and the per-row flags.
    // Padding (columns past n, rows past the tile) packs as demand 1: no DP
    // step reads it, and the tile minimum then tells whether a real demand
    // is zero.
    constexpr int LOADS = WPI * PER / 4;
    int mn = 1, mx = 0;
    for (int w0 = 0; w0 < words; w0 += WPI) {
      int4 x[LOADS];
#pragma unroll
      for (int k = 0; k < LOADS; ++k) {
        const int c = w0 * PER + 4 * k;
        x[k] = (live && c < n) ? ld_v4(row + c) : make_int4(1, 1, 1, 1);
      }
#pragma unroll
      for (int k = 0; k < LOADS; ++k) {
        mn = __vimin3_s32(mn, x[k].x, x[k].y);
        mn = __vimin3_s32(mn, x[k].z, x[k].w);
        mx = __vimax3_s32(mx, x[k].x, x[k].y);
        mx = __vimax3_s32(mx, x[k].z, x[k].w);
      }
      const int* xv = reinterpret_cast<const int*>(x);
      uint32_t pk[WPI];
#pragma unroll
      for (int k = 0; k < WPI; ++k) pk[k] = pack_raw<QT>(xv + k * PER);
#pragma unroll
      for (int k = 0; k < WPI; k += 4)
        if (w0 + k < words) tmem_st4(taddr + w0 + k, pk[k], pk[k + 1], pk[k + 2], pk[k + 3]);
    }
    tmem_wait_st();
    if (!__any_sync(0xffffffffu, mn < 0 || mx > Q)) {
      TileFlags t;
      t.inf_rows = 0u;
      t.zero = __any_sync(0xffffffffu, mn <= 0);
      t.neg = false;
      t.small_loads = !__any_sync(0xffffffffu, n * mx >= 65536);  // n <= 512, mx <= Q
      return t;
    }
  }
  // General pass: clamp to [0, Q + 1] and flag rows with a demand above Q.
  if (vec) {
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
#pragma unroll
      for (int k = 0; k < WPI; k += 4)
        if (w0 + k < words) tmem_st4(taddr + w0 + k, pk[k], pk[k + 1], pk[k + 2], pk[k + 3]);
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
  t.zero = __any_sync(0xffffffffu, zero && live);
  t.neg = __any_sync(0xffffffffu, neg && live);
  t.small_loads = false;
  return t;
}

// Output modes of the DP
constexpr int kOutNone = 0;    // cost only (batched plans)
constexpr int kOutStream = 1;  // predecessors streamed out every 16 positions
constexpr int kOutDirect = 3;  // predecessors stored by each lane, 4 per store
constexpr int kOutDelta = 2;   // i - pred(i) written in place over the consumed
                               // demand byte (on-chip backtrack of the adjoint)
constexpr int kOutDeltaLane = 4;  // i - pred(i) packed 4 (uint8) or 2 (uint16)
                                  // per word into a [word][lane] scratch

// Ring bytes per warp: RING entries x 32 lanes of an 8-byte (psi, prefix load)
// pair and a 16-bit position.
__host__ __device__ constexpr size_t ring_bytes(int ring) { return (size_t)ring * 32 * 10; }

// Deque state of one scenario (see the file comment): ring[head .. tail) in
// shared memory ([entry][lane] layout), the front and the back's psi in
// registers.  Prefix loads are kept mod 2^32: every difference taken is a
// route load below 2^32, so unsigned subtraction is exact.  Each DP step is
// split into phases so that several scenarios of a lane can be interleaved.
//  - An empty deque has bpsi = -inf, so "pop the back" is a single compare.
//  - The front registers are refreshed by the back phase when it empties the
//    deque (the new entry becomes the front), and start as entry p = 0.
//  - Without over-capacity demands in the tile (CHECK false) the newest entry
//    (route s_i alone, load q_i <= Q) never pops, so the straight-line first
//    front pop needs no size test.  The pop loop keeps it: every loop here ends
//    after at most n iterations whatever the data (rows of idle lanes may hold
//    stale values).
// PACKED (every prefix load of the tile below 2^16): an entry is one 8-byte
// word pair (psi bits, L(p) << 16 | p) and the position ring is unused.
template <int RING, bool PACKED = false>
struct DequeState {
  uint2* rpl;         // (psi bits, prefix load L(p)) of this scenario's ring (+lane)
  uint16_t* ridx;     // position p of each entry
  int head, tail, maxcnt, fidx;
  uint32_t L, fL;     // prefix load through the current position, at the front
  float K, bpsi, fpsi;
  // soft capacity: the best expired entry, c = psi(p) - beta L(p) and its p
  float cmin;
  int cidx;

  __device__ __forceinline__ void init(uint2* ring_pl, uint16_t* ring_idx, int lane,
                                       float psi0) {
    rpl = ring_pl + lane;
    ridx = ring_idx + lane;
    head = tail = maxcnt = fidx = 0;
    L = fL = 0u;
    K = 0.f;
    bpsi = -CUDART_INF_F;
    fpsi = psi0;  // entry p = 0, pushed by the first step
    cmin = CUDART_INF_F;
    cidx = -1;
  }
  __device__ __forceinline__ bool back_needed(float psi) const { return bpsi > psi; }
  __device__ __forceinline__ void pop_back() {
    --tail;
    bpsi = tail > head ? __uint_as_float(rpl[((tail - 1) & (RING - 1)) * 32].x) : -CUDART_INF_F;
  }
  __device__ __forceinline__ void back_more(float psi) {
    while (back_needed(psi)) pop_back();
  }
  // after the back pops: an emptied deque's front is the entry pushed next
  __device__ __forceinline__ void refront(float psi, int i) {
    if (tail == head) {
      fpsi = psi;
      fL = L;
      fidx = i - 1;
    }
  }
  // push p = i-1 (an equal psi stays behind the older entry: smallest p wins)
  __device__ __forceinline__ void push(float psi, int i) {
    const int slot = (tail & (RING - 1)) * 32;
    if (PACKED) {
      rpl[slot] = make_uint2(__float_as_uint(psi), __byte_perm((uint32_t)(i - 1), L, 0x5410));
    } else {
      rpl[slot] = make_uint2(__float_as_uint(psi), L);
      ridx[slot] = (uint16_t)(i - 1);
    }
    ++tail;
    bpsi = psi;
    maxcnt = max(maxcnt, tail - head);
  }
  __device__ __forceinline__ void pop_front() {
    ++head;
    const int h = (head & (RING - 1)) * 32;
    const uint2 v = rpl[h];
    fpsi = __uint_as_float(v.x);
    if (PACKED) {
      fL = v.y >> 16;
      fidx = (int)(v.y & 0xFFFFu);
    } else {
      fL = v.y;
      fidx = (int)ridx[h];
    }
  }
  template <bool CHECK>
  __device__ __forceinline__ bool front_needed(int Q) const {
    return (!CHECK || tail - head > 1) && L - fL > (uint32_t)Q;
  }
  // extend the window to customer s_i, first front pop; true if more needed
  template <bool CHECK>
  __device__ __forceinline__ bool front1(int q, int Q) {
    L += (uint32_t)q;
    const bool pf = front_needed<CHECK>(Q);
    if (pf) pop_front();
    return pf && front_needed<CHECK>(Q);
  }
  __device__ __forceinline__ void front_more(int Q) {
    while (front_needed<true>(Q)) pop_front();
  }
  // Soft capacity: every entry whose route p+1..i exceeds Q leaves the deque
  // (the newest one too, when q_i > Q) and joins the expired set, whose
  // candidate at position i is c(p) + beta (L(i) - Q); the best one is
  // c(p) = psi(p) - beta L(p) minimal (entries expire in increasing p, so "<"
  // keeps the smallest p on ties).  An emptied deque has fpsi = +inf.
  __device__ __forceinline__ void front_soft(int q, int Q, float beta) {
    L += (uint32_t)q;
    while (tail > head && L - fL > (uint32_t)Q) {
      const float c = __fsub_rn(fpsi, __fmul_rn(beta, (float)fL));
      if (c < cmin) {
        cmin = c;
        cidx = fidx;
      }
      if (tail - head > 1) {
        pop_front();
      } else {
        ++head;
        fpsi = CUDART_INF_F;
        bpsi = -CUDART_INF_F;
      }
    }
  }
  // min(window minimum, best expired candidate); ties go to the expired
  // entry (the smaller p)
  __device__ __forceinline__ float soft_best(int Q, float beta, int* idx) const {
    float best = fpsi;
    *idx = fidx;
    if (cmin < CUDART_INF_F) {
      const float c2 = __fadd_rn(__fmul_rn(beta, (float)(int)(L - (uint32_t)Q)), cmin);
      if (c2 <= best) {
        best = c2;
        *idx = cidx;
      }
    }
    return best;
  }
};

// Compact deque step for tiles without a demand above Q (hard capacity), one
// scenario per lane.  Same deque as DequeState (pop from the back every entry
// with a larger psi, push p = i-1, pop from the front every entry whose route
// exceeds Q; the front is the argmin, smallest p on ties), with fewer
// instructions and a shorter dependent chain per position:
//   - an entry is (psi, L(p) * 2^16 + p) and the lane keeps
//     Lent = L(i) * 2^16 + i, so the new entry is the previous Lent and
//     "route p+1..i exceeds Q" is (Lent - ent) > Q * 2^16 + 65535 (mod 2^32):
//     exact because the prefix loads of the entries tested differ by at most
//     2Q < 2^16 and i - p < 2^16; the low 16 bits of the front entry are the
//     predecessor, those of Lent - front the distance i - pred(i);
//   - a new psi below the front's (the deque's minimum) pops every entry: the
//     deque restarts at the new entry, so the back-pop loop needs no
//     emptiness test (it stops at the front at the latest);
//   - ring slots are byte offsets (multiples of 256: 32 lanes x 8 bytes) into
//     a [RING][32] ring of 8-byte entries.
// The newest entry (route s_i alone, load q_i <= Q) never pops from the
// front, so neither loop can empty the deque.  A scenario whose deque
// outgrows the ring is recomputed (split_rescue.cu).
template <int RING>
struct FastDeque {
  unsigned char* lb;   // this lane's slot 0 of the ring
  uint32_t head, tail; // byte offsets of the front and of the next free slot
  uint32_t Lent;       // L(i) * 2^16 + i
  uint32_t fent;       // front entry: L(p) * 2^16 + p
  bool ovf;            // the deque outgrew the ring
  float K, fpsi, bpsi;
  static constexpr uint32_t kSlots = (uint32_t)(RING - 1) << 8;
  __device__ __forceinline__ uint2* at(uint32_t off) const {
    return reinterpret_cast<uint2*>(lb + (off & kSlots));
  }
  __device__ __forceinline__ void init(uint2* ring_pl, int lane) {
    lb = reinterpret_cast<unsigned char*>(ring_pl + lane);
    head = tail = 0u;
    Lent = fent = 0u;
    ovf = false;
    K = 0.f;
    fpsi = CUDART_INF_F;  // the first step restarts the deque at entry p = 0
    bpsi = -CUDART_INF_F;
  }
  // position i with demand q16 = q_i << 16 and record (a_i, ce_i)
  __device__ __forceinline__ void step(uint32_t q16, float a, float ce, uint32_t Qc) {
    const float psi = __fadd_rn(K, a);  // psi(i-1)
    const uint32_t ent = Lent;          // (L(i-1), i-1)
    Lent += q16 + 1u;
    const bool restart = psi < fpsi;
    if (restart) {
      tail = head;
      fpsi = psi;
      fent = ent;
      bpsi = -CUDART_INF_F;
    }
    while (bpsi > psi) {
      tail -= 256u;
      bpsi = __uint_as_float(at(tail - 256u)->x);
    }
    // A full ring would overwrite the front: the scenario is flagged (its
    // results are recomputed) and its deque restarts at the new entry, so the
    // ring always holds the deque it describes and both loops end.
    if (tail - head == (uint32_t)RING * 256u) {
      ovf = true;
      head = tail;
      fpsi = psi;
      fent = ent;
    }
    *at(tail) = make_uint2(__float_as_uint(psi), ent);
    tail += 256u;
    bpsi = psi;
    while (Lent - fent > Qc) {
      head += 256u;
      const uint2 e = *at(head);
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
    K = __fadd_rn(fpsi, ce);
  }
  __device__ __forceinline__ bool overflow() const { return ovf; }
};

// TMEM demands fetched a group of G positions at a time: the loads of group
// g + 1 are issued right after the wait for group g, so each
// tcgen05.wait::ld (which waits for all of the thread's outstanding loads)
// covers G steps and finds its loads long complete.  cs[k] (shared) = TMEM
// column of position k + 1 << 16 | the tmem_rec16 selector; the array holds
// copies of position n up to index n + 2G.
template <int G>
struct TmemGroup {
  uint32_t taddr;
  const uint32_t* cs;
  uint32_t wc[G], sc[G];  // current group: words, selectors
  uint32_t wn[G], sn[G];  // next group (in flight)
  __device__ __forceinline__ void issue(int k0) {  // positions k0 + 1 .. k0 + G
#pragma unroll
    for (int u = 0; u < G; u += 4) {
      const uint4 v = *reinterpret_cast<const uint4*>(cs + k0 + u);
      const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sn[u + e] = x[e];
        wn[u + e] = tmem_ld1(taddr + (x[e] >> 16));
      }
    }
  }
  __device__ __forceinline__ void wait() {
    __syncwarp();  // the deque loops diverge; tcgen05 ops need the whole warp
    if (G == 8) {
      asm volatile("tcgen05.wait::ld.sync.aligned;"
                   : "+r"(wn[0]), "+r"(wn[1]), "+r"(wn[2 % G]), "+r"(wn[3 % G]), "+r"(wn[4 % G]),
                     "+r"(wn[5 % G]), "+r"(wn[6 % G]), "+r"(wn[7 % G])::"memory");
    } else {
      asm volatile("tcgen05.wait::ld.sync.aligned;"
                   : "+r"(wn[0]), "+r"(wn[1 % G]), "+r"(wn[2 % G]), "+r"(wn[3 % G])::"memory");
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      wc[u] = wn[u];
      sc[u] = sn[u];
    }
  }
  __device__ __forceinline__ uint32_t q16(int u) const { return __byte_perm(wc[u], 0u, sc[u]); }
};

// TMEM row with the demand returned at bits 16..31 (the record's pad is the
// byte-permute selector that puts it there; see tmem_rec16).
struct TmemQ16 {
  uint32_t taddr;
  uint32_t word;
  __device__ __forceinline__ void prefetch(const StepRec& r) { word = tmem_ld1(taddr + r.col); }
  __device__ __forceinline__ uint32_t take(const StepRec& r) {
    __syncwarp();  // the deque loops diverge; tcgen05 ops need the whole warp
    tmem_wait_ld(word);
    return __byte_perm(word, 0u, r.pad);
  }
};

// Predecessor stage: [NS * 32 rows][kBatch positions] with an odd word pitch,
// so the per-step writes of the 32 lanes (one row each) hit 32 banks.
template <typename PT>
__host__ __device__ constexpr int stage_pitch() {
  return sizeof(PT) == 2 ? kBatch + 2 : kBatch + 1;  // 9 or 17 words
}

// Rows x positions [i0, i0 + cnt) of the stage -> coalesced row segments of
// the [S, n] predecessor array.  uint16 pairs go out as 32-bit stores when
// every segment starts on 4 bytes (n even, aligned base): 8 lanes per row.
template <typename PT>
__device__ __forceinline__ void flush_stage(const PT* stage, PT* pred_tile, int n, int i0,
                                            int cnt, int rows, bool pairs, int lane) {
  constexpr int P = stage_pitch<PT>();
  __syncwarp();
  if (sizeof(PT) == 2 && pairs) {
    const int k = lane & 7, r0 = lane >> 3;  // pair k of row r0 + 4j
    if (2 * k < cnt) {
      const uint32_t* sp = reinterpret_cast<const uint32_t*>(stage) + r0 * (P / 2) + k;
      uint32_t* dst = reinterpret_cast<uint32_t*>(pred_tile + (int64_t)r0 * n + (i0 - 1)) + k;
      const int64_t step = 2 * (int64_t)n;  // 4 rows, in 32-bit words
#pragma unroll 4
      for (int r = r0; r < rows; r += 4) {
        *dst = *sp;
        sp += 4 * (P / 2);
        dst += step;
      }
    }
  } else {
    const int k = lane & 15, r0 = lane >> 4;  // position k of row r0 + 2j
    if (k < cnt) {
      const PT* sp = stage + r0 * P + k;
      PT* dst = pred_tile + (int64_t)r0 * n + (i0 - 1) + k;
      const int64_t step = 2 * (int64_t)n;
#pragma unroll 4
      for (int r = r0; r < rows; r += 2) {
        *dst = *sp;
        sp += 2 * P;
        dst += step;
      }
    }
  }
  __syncwarp();
}

// The DP of NS scenarios per lane (see the file comment).  Every lane of the
// warp runs it (lanes beyond the tile on stale data, outputs dropped) so that
// TMEM loads and the 16-position output batches stay warp-collective.
// Scenario s of the lane is tile row s * 32 + lane.
// CHECK: the tile holds a scenario with a demand above Q; first_inf records
// the first such position of each scenario.
// REC_SHARED: rec points to shared memory (loaded as LDS.128) and holds copies
// of position n at indices n and n + 1.  Records are loaded two positions
// ahead, so the TMEM load of the next demand reads a column loaded a step
// earlier instead of waiting for this step's shared load (1.603 -> 1.589 ms
// at n = 500, S = 10^6).  Records read from global memory stay one position
// ahead: two ahead slowed the batched shared-memory kernel by 4%.
// OUT == kOutStream: predecessors through the shared-memory stage (any n);
// OUT == kOutDirect: each lane stores its own row, 4 positions per 8-byte
// (uint16) or 16-byte (int32) store, when n % 4 == 0 and the rows are aligned
// -- no stage, and 4 row segments complete a 32-byte sector.
// OUT == kOutDelta (NS = 1, shared-memory row): i - pred(i) overwrites the
// consumed demand byte of customer s_i.
// UNR: unroll factor of the position loop (1 where registers are tight).
// PACKED: every prefix load of the tile is below 2^16 (see DequeState).
template <int NS, typename QT, typename PT, int RING, int OUT, bool CHECK, bool REC_SHARED,
          typename SRC, int UNR = 2, bool PACKED = false, bool SOFT = false>
__device__ __forceinline__ void dp_rows(SRC* src, QT* row, int n, int Q, const StepRec* rec,
                                        uint2* ring_pl, uint16_t* ring_idx, int lane,
                                        PT* stage, PT* pred_tile, int rows, bool check_delta,
                                        uint32_t* first_inf, bool* bad, float* K_out,
                                        float beta = 0.f, uint32_t* dout = nullptr) {
  constexpr int kP = stage_pitch<PT>();
  constexpr int kPer = 4 / (int)sizeof(QT);  // deltas per word (kOutDeltaLane)
  uint32_t dlast = 0u;
  const uint32_t rec_s = REC_SHARED ? (uint32_t)__cvta_generic_to_shared(rec) : 0u;
  auto load_rec = [&](int k) -> StepRec {
    if (REC_SHARED) return ld_rec_shared(rec_s + 16u * (uint32_t)k);
    return ld_rec_any(rec + k);
  };
  StepRec rn = load_rec(0);
  StepRec rn2 = REC_SHARED ? load_rec(1) : rn;
  DequeState<RING, PACKED> st[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s)
    st[s].init(ring_pl + s * RING * 32, ring_idx + s * RING * 32, lane, __fadd_rn(0.f, rn.a));
#pragma unroll
  for (int s = 0; s < NS; ++s) src[s].prefetch(rn);

  // One DP step at position i; p[s] = pred(i) of scenario s (-1 once infeasible).
  auto step = [&](int i, int* p) {
    const StepRec r = rn;
    int q[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) q[s] = src[s].take(r);
    // next position's demand (its record came a step ago), the record after it
    if (REC_SHARED) {
      rn = rn2;
      rn2 = load_rec(i + 1);
    } else {
      rn = load_rec(min(i, n - 1));
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) src[s].prefetch(rn);
    // Each lane pops on its own: warp votes that skipped the pop phases when
    // no lane needed them were measured slower (1.77 ms against 1.61 ms at
    // n = 500, S = 10^6) -- a vote waits for the whole warp to reconverge.
    float psi[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      psi[s] = __fadd_rn(st[s].K, r.a);
      st[s].back_more(psi[s]);
      st[s].refront(psi[s], i);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      st[s].push(psi[s], i);
      if (SOFT) {
        st[s].front_soft(q[s], Q, beta);
      } else {
        if (CHECK && q[s] > Q && first_inf[s] > (uint32_t)n) first_inf[s] = (uint32_t)i;
        st[s].template front1<CHECK>(q[s], Q);
        st[s].front_more(Q);
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (SOFT) {
        int idx;
        st[s].K = __fadd_rn(st[s].soft_best(Q, beta, &idx), r.ce);
        p[s] = idx;
        continue;
      }
      st[s].K = __fadd_rn(st[s].fpsi, r.ce);
      p[s] = (CHECK && (uint32_t)i >= first_inf[s]) ? -1 : st[s].fidx;
      if (OUT == kOutDelta) {
        const uint32_t delta = (uint32_t)(i - st[s].fidx);
        if (check_delta && delta > (sizeof(QT) == 1 ? 255u : 65535u)) bad[s] = true;
        row[r.col] = (QT)delta;
      }
      if (OUT == kOutDeltaLane) dlast = (uint32_t)(i - st[s].fidx);  // NS = 1
    }
  };

  if (OUT == kOutDeltaLane) {
    // position j's delta sits in word (j - 1) / kPer at slot (j - 1) % kPer;
    // whole words first (static slots), then the last partial word
    constexpr int kBits = 8 * (int)sizeof(QT);
    uint32_t any = 0u;  // OR of the deltas: one range test per row
    int i = 1;
    for (; i + kPer - 1 <= n; i += kPer) {
      uint32_t w = 0u;
      int p;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        step(i + u, &p);
        any |= dlast;
        w |= dlast << (kBits * u);
      }
      dout[((i - 1) / kPer) * 32] = w;
    }
    if (i <= n) {
      uint32_t w = 0u;
      int p;
      for (int u = 0; i + u <= n; ++u) {
        step(i + u, &p);
        any |= dlast;
        w |= dlast << (kBits * u);
      }
      dout[((i - 1) / kPer) * 32] = w;
    }
    if (check_delta && any > (sizeof(QT) == 1 ? 255u : 65535u)) bad[0] = true;
  } else if (OUT == kOutDirect) {
    PT* prow[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) prow[s] = pred_tile + (int64_t)(s * 32 + lane) * n;
    for (int i = 1; i <= n; i += 4) {
      int p[4][NS];
#pragma unroll
      for (int u = 0; u < 4; ++u) step(i + u, p[u]);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (s * 32 + lane < rows) {
          if (sizeof(PT) == 2) {
            *reinterpret_cast<uint2*>(prow[s] + (i - 1)) =
                make_uint2(__byte_perm(p[0][s], p[1][s], 0x5410),
                           __byte_perm(p[2][s], p[3][s], 0x5410));
          } else {
            *reinterpret_cast<int4*>(prow[s] + (i - 1)) =
                make_int4(p[0][s], p[1][s], p[2][s], p[3][s]);
          }
        }
      }
    }
  } else {
    const bool pairs = sizeof(PT) == 2 && (n & 1) == 0 &&
                       (reinterpret_cast<uintptr_t>(pred_tile) & 3) == 0;
    for (int i0 = 1; i0 <= n; i0 += kBatch) {
      const int ie = min(n, i0 + kBatch - 1);
#pragma unroll UNR
      for (int i = i0; i <= ie; ++i) {
        int p[NS];
        step(i, p);
        if (OUT == kOutStream) {
#pragma unroll
          for (int s = 0; s < NS; ++s) stage[(s * 32 + lane) * kP + (i - i0)] = (PT)p[s];
        }
      }
      if (OUT == kOutStream)
        flush_stage<PT>(stage, pred_tile, n, i0, ie - i0 + 1, rows, pairs, lane);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    bad[s] |= st[s].maxcnt > RING;
    K_out[s] = st[s].K;
  }
}

// The DP of one scenario per lane with FastDeque steps, for tiles without a
// demand above Q, rows in TMEM, demands fetched KG positions ahead
// (TmemGroup; cs as there), records (a_i, ce_i) from shared memory.  Every
// lane of the warp runs it (lanes beyond the tile on stale data, outputs
// dropped).
// OUT == kOutNone: cost only; kOutDirect: predecessors stored by each lane, 4
// positions per store (n % 4 == 0, aligned rows); kOutDeltaLane: i - pred(i)
// packed 4 (uint8) or 2 (uint16) per word into the [word][lane] scratch dout
// (check_delta: a tile with zero demands, where a route may be longer than
// the staging type holds).
// G = 8 positions per group where registers allow (16 warps per SM), else 4.
constexpr int kGroup = 8;
template <typename QT, typename PT, int RING, int OUT, int G = kGroup>
__device__ __forceinline__ void dp_fast(uint32_t taddr, const uint32_t* cs, int n, int Q,
                                        const StepRec* rec, uint2* ring_pl, int lane,
                                        PT* pred_tile, int rows, bool check_delta, bool* bad,
                                        float* K_out, uint32_t* dout) {
  constexpr int kPer = 4 / (int)sizeof(QT);  // deltas per word (kOutDeltaLane)
  constexpr int kBits = 8 * (int)sizeof(QT);
  constexpr uint32_t kLow = sizeof(QT) == 1 ? 0xFFu : 0xFFFFu;
  const uint32_t Qc = ((uint32_t)Q << 16) | 0xFFFFu;
  const uint32_t rec_s = (uint32_t)__cvta_generic_to_shared(rec);
  FastDeque<RING> st;
  st.init(ring_pl, lane);
  TmemGroup<G> tg;
  tg.taddr = taddr;
  tg.cs = cs;
  tg.issue(0);
  tg.wait();
  tg.issue(G);
  const bool live = lane < rows;
  PT* prow = (OUT == kOutDirect) ? pred_tile + (int64_t)lane * n : nullptr;
  uint32_t any = 0u;   // OR of the deltas (kOutDeltaLane): one range test per row
  uint32_t f[4];       // last four front entries (kOutDirect)
  uint32_t dw = 0u;    // delta word being packed (kOutDeltaLane)
  const int ng = (n + G - 1) / G;
  for (int g = 0; g < ng; ++g) {
    const int i0 = g * G + 1;
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int i = i0 + u;
      if (G * (g + 1) > n && i > n) break;  // ragged last group
      const StepRec r = ld_rec_shared(rec_s + 16u * (uint32_t)(i - 1));
      st.step(tg.q16(u), r.a, r.ce, Qc);
      if (OUT == kOutDirect) {
        f[u & 3] = st.fent;
        if ((u & 3) == 3 && live) {
          if (sizeof(PT) == 2) {
            *reinterpret_cast<uint2*>(prow + (i - 4)) =
                make_uint2(__byte_perm(f[0], f[1], 0x5410), __byte_perm(f[2], f[3], 0x5410));
          } else {
            *reinterpret_cast<int4*>(prow + (i - 4)) =
                make_int4((int)(f[0] & 0xFFFFu), (int)(f[1] & 0xFFFFu), (int)(f[2] & 0xFFFFu),
                          (int)(f[3] & 0xFFFFu));
          }
        }
      } else if (OUT == kOutDeltaLane) {
        const uint32_t dl = (st.Lent - st.fent) & 0xFFFFu;  // i - pred(i)
        if (check_delta) any |= dl;
        const int sl = (i - 1) % kPer;
        dw = (sl == 0 ? 0u : dw) | ((dl & kLow) << (kBits * sl));
        if (sl == kPer - 1 || i == n) dout[((i - 1) / kPer) * 32] = dw;
      }
    }
    tg.wait();
    tg.issue((g + 2) * G);
  }
  tg.wait();  // the look-ahead group past the row
  *bad |= st.overflow() || (check_delta && any > (sizeof(QT) == 1 ? 255u : 65535u));
  *K_out = st.K;
}

}  // namespace

// ------------------------------------------------------------------ kernels
template <typename PT, int NS>
__host__ __device__ constexpr size_t stage_bytes_of() {
  return (((size_t)NS * 32 * stage_pitch<PT>() * sizeof(PT)) + 15) & ~(size_t)15;
}

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
  const size_t stage_bytes = OUT == kOutStream ? stage_bytes_of<PT, 1>() : 0;
  const size_t per_warp = (size_t)32 * row_stride + ring_bytes(RING) + stage_bytes;
  unsigned char* wbase = smem + off + per_warp * warp;
  QT* qb = reinterpret_cast<QT*>(wbase);
  uint2* ring_pl = reinterpret_cast<uint2*>(wbase + (size_t)32 * row_stride);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + RING * 32);
  PT* stage = reinterpret_cast<PT*>(ring_idx + RING * 32);
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
    __syncwarp();

    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    float K;
    QT* row = qb + lane * rs_elems;
    PT* pred_tile = a.pred ? reinterpret_cast<PT*>(a.pred) + s0 * n : nullptr;
    const bool valid = lane < rows;
    SmemQ<QT> src{row, 0};
    if (tf.inf_rows)
      dp_rows<1, QT, PT, RING, OUT, true, false>(&src, row, n, Q, rec, ring_pl, ring_idx, lane,
                                                 stage, pred_tile, pred_tile ? rows : 0, tf.zero,
                                                 &first_inf, &bad, &K);
    else
      dp_rows<1, QT, PT, RING, OUT, false, false>(&src, row, n, Q, rec, ring_pl, ring_idx,
                                                  lane, stage, pred_tile, pred_tile ? rows : 0,
                                                  tf.zero, &first_inf, &bad, &K);
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
// (its dynamic shared memory request guarantees it) allocates all 512 TMEM
// columns; warp w holds its tile in lane quadrant w % 4, column block w / 4
// of cols_per_warp columns.  XW sizes the launch bounds (512 + 32 XW
// threads): the default launch has 16 warps (XW = 0, two steps per loop
// iteration); the wide one 17..24 (XW = 8, fewer columns each, 80 registers a
// thread: one step per iteration, smaller ingest batches), taken when that
// many finish every tile in one round.
template <typename QT, typename PT, int RING, int OUT, int XW>
__global__ void __launch_bounds__(512 + 32 * XW, 1) split_tmem_kernel(SplitDequeArgs a,
                                                                     int64_t tiles,
                                                                     int cols_per_warp) {
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
  // tour records in shared memory (a row that fits a warp's TMEM columns has
  // n <= 512), plus a copy of position n after them
  StepRec* rec = reinterpret_cast<StepRec*>(smem);
  for (int k = threadIdx.x; k <= n + 1; k += blockDim.x) rec[k] = tmem_rec16<QT>(a.rec[min(k, n - 1)]);
  // from the records in global memory: the shared copy above is not
  // complete until the barrier below
  uint32_t* cs = reinterpret_cast<uint32_t*>(rec + n + 2);
  for (int k = threadIdx.x; k < n + 3 * kGroup; k += blockDim.x) {
    const StepRec r = tmem_rec16<QT>(a.rec[min(k, n - 1)]);
    cs[k] = (r.col << 16) | r.pad;
  }
  const size_t off = ((size_t)n + 2) * sizeof(StepRec) + cs_bytes(n);
  const size_t stage_bytes = OUT == kOutStream ? stage_bytes_of<PT, 1>() : 0;
  const size_t per_warp = ring_bytes(RING) + stage_bytes;
  unsigned char* wbase = smem + off + per_warp * warp;
  uint2* ring_pl = reinterpret_cast<uint2*>(wbase);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + RING * 32);
  PT* stage = reinterpret_cast<PT*>(ring_idx + RING * 32);
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
    const int32_t* tsrc = a.demands + s0 * n;
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    float K;
    PT* pred_tile = a.pred ? reinterpret_cast<PT*>(a.pred) + s0 * n : nullptr;
    const int prow = pred_tile ? rows : 0;
    constexpr int UNR = XW == 0 ? 2 : 1;
    using Src = TmemQ<QT, true>;
    const TileFlags tf = ingest_tile_tmem<QT, XW == 0 ? 16 : 8>(tsrc, rows, n, Q, taddr, lane);
    if (tf.inf_rows) {
      Src src{taddr, 0u};
      dp_rows<1, QT, PT, RING, OUT, true, true, Src, UNR>(
          &src, (QT*)nullptr, n, Q, rec, ring_pl, ring_idx, lane, stage, pred_tile, prow,
          false, &first_inf, &bad, &K);
    } else if (OUT == kOutStream) {  // predecessors through the stage (n % 4 != 0)
      Src src{taddr, 0u};
      dp_rows<1, QT, PT, RING, OUT, false, true, Src, UNR>(
          &src, (QT*)nullptr, n, Q, rec, ring_pl, ring_idx, lane, stage, pred_tile, prow,
          false, &first_inf, &bad, &K);
    } else {
      dp_fast<QT, PT, RING, OUT, XW == 0 ? 8 : 4>(taddr, cs, n, Q, rec, ring_pl, lane,
                                                  pred_tile, prow, false, &bad, &K, nullptr);
    }
    neg |= tf.neg;
    const bool valid = lane < rows;
    bad = bad && valid;
    if (valid) {
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else if (a.cost) {
        a.cost[s0 + lane] = first_inf <= (uint32_t)n ? CUDART_INF_F : (float)((double)K + Dn);
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

// Fused adjoint with TMEM staging: the forward DP of split_tmem_kernel
// (cost not stored), i - pred(i) of each position packed into the warp's
// slot of a [word][lane] global scratch (one coalesced 128-byte store every
// 4 uint8 / 2 uint16 positions), then each lane walks its own scenario's
// optimal routes back from position n and counts route starts / ends in
// shared-memory histograms.  The CTA holds blockDim.x / 32 = 16..24 warps:
// more than 16 when that many take every tile in one round where 16 would
// need two (a second, partly empty round costs a whole row's time).  Warp w
// holds its tile in TMEM lane quadrant w % 4, column block w / 4 of
// cols_per_warp.
template <typename QT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) split_tmem_adj_kernel(SplitDequeArgs a,
                                                                 int64_t tiles,
                                                                 int cols_per_warp,
                                                                 uint32_t* dscratch) {
  constexpr int RING = 16;
  constexpr int kPer = 4 / (int)sizeof(QT);
  constexpr int UNR = MAXT <= 512 ? 2 : 1;  // 21..24 warps leave 80 registers
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  const int n = a.n, Q = a.Q;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int dwords = (n + kPer - 1) / kPer;

  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  StepRec* rec = reinterpret_cast<StepRec*>(smem);
  for (int k = threadIdx.x; k <= n + 1; k += blockDim.x) rec[k] = tmem_rec16<QT>(a.rec[min(k, n - 1)]);
  // from the records in global memory: the shared copy above is not
  // complete until the barrier below
  uint32_t* cs = reinterpret_cast<uint32_t*>(rec + n + 2);
  for (int k = threadIdx.x; k < n + 3 * kGroup; k += blockDim.x) {
    const StepRec r = tmem_rec16<QT>(a.rec[min(k, n - 1)]);
    cs[k] = (r.col << 16) | r.pad;
  }
  size_t off = ((size_t)n + 2) * sizeof(StepRec) + cs_bytes(n);
  unsigned int* hist_sm = reinterpret_cast<unsigned int*>(smem + off);
  off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
  for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x) hist_sm[k] = 0u;
  uint2* ring_pl = reinterpret_cast<uint2*>(smem + off + ring_bytes(RING) * warp);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + RING * 32);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) +
                         (uint32_t)((warp >> 2) * cols_per_warp);
  uint32_t* dl = dscratch + ((int64_t)blockIdx.x * nwarps + warp) * dwords * 32 + lane;

  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;
  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  for (int64_t tile = (int64_t)blockIdx.x * nwarps + warp; tile < tiles; tile += wstride) {
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    float K;
    using Src = TmemQ<QT, true>;
    const TileFlags tf =
        ingest_tile_tmem<QT, MAXT <= 512 ? 16 : 8>(a.demands + s0 * n, rows, n, Q, taddr, lane);
    if (tf.inf_rows) {
      Src src{taddr, 0u};
      dp_rows<1, QT, int32_t, RING, kOutDeltaLane, true, true, Src, UNR>(
          &src, (QT*)nullptr, n, Q, rec, ring_pl, ring_idx, lane, nullptr, nullptr, 0, tf.zero,
          &first_inf, &bad, &K, 0.f, dl);
    } else {
      dp_fast<QT, int32_t, RING, kOutDeltaLane, MAXT <= 512 ? 8 : 4>(
          taddr, cs, n, Q, rec, ring_pl, lane, nullptr, 0, tf.zero, &bad, &K, dl);
    }
    neg |= tf.neg;
    const bool valid = lane < rows;
    bad = bad && valid;
    if (bad) {
      const uint32_t k = atomicAdd(a.fb_count, 1u);
      a.fb_list[k] = (uint32_t)(s0 + lane);
    }
    any_inf |= tf.inf_rows;
    any_fb |= __ballot_sync(0xffffffffu, bad);
    // backtrack of this lane's scenario through its own deltas (written by
    // this thread above: program order makes them visible)
    if (valid && !bad && first_inf > (uint32_t)n) {
      for (int i = n; i > 0;) {
        const uint32_t w = dl[((i - 1) / kPer) * 32];
        const int sh = 8 * (int)sizeof(QT) * ((i - 1) % kPer);
        const int d = (int)((w >> sh) & (sizeof(QT) == 1 ? 0xFFu : 0xFFFFu));
        if (d < 1 || d > i) break;  // 1 <= i - pred(i) <= i; keeps the walk bounded
        const int p = i - d;
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
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, 512);
  for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x)
    if (hist_sm[k]) atomicAdd(&a.hist[k], (unsigned long long)hist_sm[k]);
}

// Soft-capacity Split with TMEM staging (16 warps per SM, as split_tmem_kernel
// with XW = 0): every split is allowed and a route pays beta per unit of
// load above Q.  Demands are staged exactly (no clamp to Q + 1); a row with a
// demand the staging type cannot hold goes to the plain kernel.
template <typename QT, typename PT, int OUT>
__global__ void __launch_bounds__(512, 1) split_tmem_soft_kernel(SplitDequeArgs a, int64_t tiles) {
  constexpr int RING = 16;
  constexpr int cols_per_warp = 128;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  const int n = a.n, Q = a.Q;
  const float beta = a.beta;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  StepRec* rec = reinterpret_cast<StepRec*>(smem);
  for (int k = threadIdx.x; k <= n + 1; k += blockDim.x) rec[k] = tmem_rec<QT>(a.rec[min(k, n - 1)]);
  const size_t off = ((size_t)n + 2) * sizeof(StepRec);
  const size_t stage_bytes = OUT == kOutStream ? stage_bytes_of<PT, 1>() : 0;
  const size_t per_warp = ring_bytes(RING) + stage_bytes;
  unsigned char* wbase = smem + off + per_warp * warp;
  uint2* ring_pl = reinterpret_cast<uint2*>(wbase);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + RING * 32);
  PT* stage = reinterpret_cast<PT*>(ring_idx + RING * 32);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) +
                         (uint32_t)((warp >> 2) * cols_per_warp);
  // the largest demand the staging type holds exactly (one below its top, so
  // the staging's own clamp never collides with a real value)
  const int cap = (sizeof(QT) == 1 ? 255 : 65535) - 1;
  const double Dn = *a.Dn;
  bool neg = false;
  uint32_t any_fb = 0;
  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  for (int64_t tile = (int64_t)blockIdx.x * nwarps + warp; tile < tiles; tile += wstride) {
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    float K;
    PT* pred_tile = a.pred ? reinterpret_cast<PT*>(a.pred) + s0 * n : nullptr;
    const int prow = pred_tile ? rows : 0;
    using Src = TmemQ<QT>;
    const TileFlags tf = ingest_tile_tmem<QT, 16>(a.demands + s0 * n, rows, n, cap, taddr, lane);
    Src src{taddr, 0u};
    if (tf.small_loads)
      dp_rows<1, QT, PT, RING, OUT, false, true, Src, 2, true, true>(
          &src, (QT*)nullptr, n, Q, rec, ring_pl, ring_idx, lane, stage, pred_tile, prow, false,
          &first_inf, &bad, &K, beta);
    else
      dp_rows<1, QT, PT, RING, OUT, false, true, Src, 2, false, true>(
          &src, (QT*)nullptr, n, Q, rec, ring_pl, ring_idx, lane, stage, pred_tile, prow, false,
          &first_inf, &bad, &K, beta);
    neg |= tf.neg;
    const bool valid = lane < rows;
    bad = (bad || ((tf.inf_rows >> lane) & 1u)) && valid;
    if (valid) {
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else if (a.cost) {
        a.cost[s0 + lane] = (float)((double)K + Dn);
      }
    }
    any_fb |= __ballot_sync(0xffffffffu, bad);
    __syncwarp();
  }
  if (lane == 0) {
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
// tours finish together.
// NS tiles of one tour per warp item (NS = 2: scenarios s0 + lane and
// s0 + 32 + lane on each lane, the two deques stepped together), rows staged
// in shared memory.
template <typename QT, int RING, int NS>
__global__ void __launch_bounds__(256, 1) split_batch_kernel(BatchKernelArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Q = a.Q;
  const int row_bytes_max = staged_row_stride(a.n_max, (int)sizeof(QT));
  const size_t per_warp = NS * ((size_t)32 * row_bytes_max + ring_bytes(RING));
  unsigned char* wbase = smem + per_warp * warp;
  QT* qb = reinterpret_cast<QT*>(wbase);  // NS blocks of 32 rows
  uint2* ring_pl = reinterpret_cast<uint2*>(wbase + (size_t)NS * 32 * row_bytes_max);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + NS * RING * 32);
  const int64_t tiles = (a.S + 31) / 32;
  const int64_t per_tour = (tiles + NS - 1) / NS;  // items per tour
  const int64_t items = per_tour * a.B;
  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;

  auto pop = [&]() -> int64_t {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(a.counter, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, k, 0);
  };
  int64_t item = pop();
  while (item < items) {
    const int b = a.order[item / per_tour];
    const int64_t s0 = (item % per_tour) * 32 * NS;
    const int n = a.n[b];
    const int rs_elems = staged_row_stride(n, (int)sizeof(QT)) / (int)sizeof(QT);
    int rows[NS];
    uint32_t tinf = 0;
    SmemQ<QT> src[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int64_t st = s0 + 32 * s;
      rows[s] = st >= a.S ? 0 : (int)imin64(32, a.S - st);
      QT* qs = qb + (size_t)s * 32 * row_bytes_max / sizeof(QT);
      if (rows[s] > 0) {
        const TileFlags tf = ingest_tile<QT>(a.demands + a.dem_off[b] + st * n, rows[s], n,
                                             rs_elems, Q, qs, lane);
        neg |= tf.neg;
        tinf |= tf.inf_rows;
      }
      src[s] = SmemQ<QT>{qs + lane * rs_elems, 0};
    }
    const int64_t next = pop();
    __syncwarp();
    uint32_t first_inf[NS];
    bool bad[NS];
    float K[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      first_inf[s] = (uint32_t)n + 1;
      bad[s] = false;
    }
    const StepRec* rec = a.rec + a.rec_off[b];
    if (tinf)
      dp_rows<NS, QT, int32_t, RING, kOutNone, true, false>(src, src[0].row, n, Q, rec, ring_pl,
                                                            ring_idx, lane, nullptr, nullptr, 0,
                                                            false, first_inf, bad, K);
    else
      dp_rows<NS, QT, int32_t, RING, kOutNone, false, false>(src, src[0].row, n, Q, rec, ring_pl,
                                                             ring_idx, lane, nullptr, nullptr, 0,
                                                             false, first_inf, bad, K);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const bool valid = lane < rows[s];
      const bool bd = bad[s] && valid;
      if (valid) {
        const int64_t g = (int64_t)b * a.S + s0 + 32 * s + lane;
        if (bd) {
          const uint32_t k = atomicAdd(a.fb_count, 1u);
          a.fb_list[k] = (unsigned long long)g;
        } else {
          a.costs[g] = first_inf[s] <= (uint32_t)n ? CUDART_INF_F
                                                     : (float)((double)K[s] + a.Dn[b]);
        }
      }
      any_fb |= __ballot_sync(0xffffffffu, bd);
    }
    any_inf |= tinf;
    __syncwarp();
    item = next;
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (neg) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  }
}

// Batched Split with TMEM staging: one CTA per SM owns all 512 TMEM columns;
// warp w holds its tile in lane quadrant w % 4, column block w / 4 of
// cols_per_warp columns (16 warps x 128, 8 x 256 or 4 x 512 columns), and
// copies the current tour's records into its own shared-memory slice.
template <typename QT, int RING>
__global__ void __launch_bounds__(512, 1) split_batch_tmem_kernel(BatchKernelArgs a,
                                                                  int cols_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Q = a.Q;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  const size_t rec_bytes = ((size_t)a.n_max + 2) * sizeof(StepRec);
  const size_t per_warp = ring_bytes(RING) + rec_bytes;
  unsigned char* wbase = smem + per_warp * warp;
  uint2* ring_pl = reinterpret_cast<uint2*>(wbase);
  uint16_t* ring_idx = reinterpret_cast<uint16_t*>(ring_pl + RING * 32);
  StepRec* rec_sm = reinterpret_cast<StepRec*>(ring_idx + RING * 32);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) +
                         (uint32_t)((warp >> 2) * cols_per_warp);
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
  int cur_b = -1;
  while (item < items) {
    const int b = a.order[item / tiles];
    const int64_t s0 = (item % tiles) * 32;
    const int n = a.n[b];
    const int rows = (int)imin64(32, a.S - s0);
    if (b != cur_b) {  // this tour's records into the warp's slice
      __syncwarp();
      const StepRec* src = a.rec + a.rec_off[b];
      for (int k = lane; k <= n + 1; k += 32) rec_sm[k] = tmem_rec<QT>(ld_rec_any(src + min(k, n - 1)));
      __syncwarp();
      cur_b = b;
    }
    const TileFlags tf =
        ingest_tile_tmem<QT>(a.demands + a.dem_off[b] + s0 * n, rows, n, Q, taddr, lane);
    neg |= tf.neg;
    const int64_t next = pop();
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    float K;
    TmemQ<QT> src{taddr, 0u};
    if (tf.inf_rows)
      dp_rows<1, QT, int32_t, RING, kOutNone, true, true>(&src, (QT*)nullptr, n, Q, rec_sm,
                                                          ring_pl, ring_idx, lane, nullptr,
                                                          nullptr, 0, false, &first_inf, &bad,
                                                          &K);
    else
      dp_rows<1, QT, int32_t, RING, kOutNone, false, true>(&src, (QT*)nullptr, n, Q, rec_sm,
                                                           ring_pl, ring_idx, lane, nullptr,
                                                           nullptr, 0, false, &first_inf, &bad,
                                                           &K);
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
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, 512);
}

// ------------------------------------------------------------------ host side
bool deque_supported(int n, int Q) { return n >= 1 && n <= 65534 && Q >= 1 && Q <= 32767; }

namespace {
int out_mode(bool hist, bool want_pred) {
  return hist ? kOutDelta : (want_pred ? kOutStream : kOutNone);
}
size_t stage_bytes_for(int pred_bytes, int ns) {
  if (pred_bytes <= 0) return 0;
  const int pitch = pred_bytes == 2 ? stage_pitch<uint16_t>() : stage_pitch<int32_t>();
  return (((size_t)ns * 32 * pitch * pred_bytes) + 15) & ~(size_t)15;
}
// TMEM single-tour launch: 16 warps with 128 TMEM columns each.  Measured at
// n = 500, S = 10^6: one scenario per lane with 16 warps (2.07 ms) beats two
// per lane with 8 warps (2.72 ms) -- the DP is bound by dependent latencies,
// which more warps hide better than two chains per thread -- and 4 more warps
// staging in shared memory (96 registers each) gained nothing.  When 17..24
// warps take every tile in one round where 16 would need two (16 to 24 tiles
// per SM) and the rows fit their share of the columns, the launch is that
// wide instead.
constexpr int kTmemColsPerWarp = 128;
constexpr int kTmemMaxWarps = 24;
constexpr int kWideXW = kTmemMaxWarps - 16;  // launch bounds of the wide kernels
constexpr size_t kMaxSmemPerCta = 227 * 1024;
// TMEM columns of each warp when nw warps share the 512 (nw / 4 rounded up
// warps per lane quadrant), in whole 4-column stores
int tmem_cols_per_warp(int nw) { return nw <= 16 ? kTmemColsPerWarp : (512 / ((nw + 3) / 4)) & ~3; }
}  // namespace

DequeConfig deque_config(int n, int Q, int warps, int ring, bool hist, int pred_bytes,
                         bool allow_tmem) {
  DequeConfig c;
  c.qbytes = Q <= 254 ? 1 : 2;
  c.ring = ring;
  c.rec_in_smem = n <= 4096;
  c.row_stride = staged_row_stride(n, c.qbytes);
  const size_t rec = c.rec_in_smem ? (size_t)n * sizeof(StepRec) : 0;
  // TMEM staging when a row fits a warp's columns and no in-place deltas are
  // needed.
  c.tmem = allow_tmem && !hist && tmem_row_words(n, c.qbytes) <= kTmemColsPerWarp;
  if (c.tmem) {
    const size_t base = ((size_t)n + 2) * sizeof(StepRec) + cs_bytes(n);
    const size_t per_warp = ring_bytes(ring) + stage_bytes_for(pred_bytes, 1);
    c.warps = 16;
    const size_t need = base + (size_t)c.warps * per_warp;
    c.smem = need > kOneCtaPerSmSmem ? need : kOneCtaPerSmSmem;
    return c;
  }
  size_t off = rec;
  if (hist) {
    off += ((size_t)n * 2 + 15) & ~(size_t)15;
    off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
  }
  const size_t stage = hist ? 0 : stage_bytes_for(pred_bytes, 1);
  const size_t per_warp = (size_t)32 * c.row_stride + ring_bytes(ring) + stage;
  // default: 4 warps per CTA, fewer when long rows would not fit
  c.warps = warps > 0 ? warps : 4;
  while (warps == 0 && c.warps > 1 && off + (size_t)c.warps * per_warp > kMaxSmemPerCta) --c.warps;
  c.smem = off + (size_t)c.warps * per_warp;
  return c;
}

DequeConfig deque_config_wide(const DequeConfig& c, int n, int Q, int64_t S, bool direct_ok,
                              int sms) {
  if (!c.tmem || c.ring != 16 || !direct_ok) return c;
  const int nw = split_tmem_adj_warps(n, Q, S, sms);
  if (nw <= 16) return c;
  DequeConfig w = c;
  w.warps = nw;
  const size_t need = ((size_t)n + 2) * sizeof(StepRec) + cs_bytes(n) + (size_t)nw * ring_bytes(16);
  w.smem = need > kOneCtaPerSmSmem ? need : kOneCtaPerSmSmem;
  return w;
}

namespace {
template <typename QT, typename PT, int RING, int OUT>
int launch_t(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
             int* occ_out) {
  if (a.soft) {  // soft capacity: TMEM staging only (checked by the caller)
    if (OUT == kOutDelta || !c.tmem) return (int)cudaErrorInvalidValue;
    const bool direct = OUT == kOutStream && (a.n & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(a.pred) & 15) == 0;
    auto k = direct ? split_tmem_soft_kernel<QT, PT, kOutDirect>
                    : split_tmem_soft_kernel<QT, PT, OUT == kOutDelta ? kOutNone : OUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem);
    if (e != cudaSuccess) return (int)e;
    if (occ_out) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_out, k, 512, c.smem);
      if (*occ_out > 1) *occ_out = 1;
      return (int)e;
    }
    k<<<grid, 512, c.smem, st>>>(a, (a.S + 31) / 32);
    return (int)cudaGetLastError();
  }
  if (OUT != kOutDelta && c.tmem) {
    // predecessors stored 4 per lane when every row segment is aligned
    const bool direct = OUT == kOutStream && (a.n & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(a.pred) & 15) == 0;
    // wide launch (17..24 warps, deque_config_wide): 16-entry rings, direct
    // or no predecessors
    const bool wide = c.warps > 16;
    if (wide && (RING != 16 || (OUT == kOutStream && !direct))) return (int)cudaErrorInvalidValue;
    auto k = wide ? (direct ? split_tmem_kernel<QT, PT, 16, kOutDirect, kWideXW>
                            : split_tmem_kernel<QT, int32_t, 16, kOutNone, kWideXW>)
                  : (direct ? split_tmem_kernel<QT, PT, RING, kOutDirect, 0>
                            : split_tmem_kernel<QT, PT, RING, OUT, 0>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem);
    if (e != cudaSuccess) return (int)e;
    if (occ_out) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_out, k, c.warps * 32, c.smem);
      if (*occ_out > 1) *occ_out = 1;  // one TMEM owner per SM
      return (int)e;
    }
    const int64_t tiles = (a.S + 31) / 32;
    k<<<grid, c.warps * 32, c.smem, st>>>(a, tiles, tmem_cols_per_warp(c.warps));
    return (int)cudaGetLastError();
  }
  const int64_t tiles = (a.S + 31) / 32;
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

// Batched launch shapes: warps > 0 = shared-memory staging with that many
// warps per CTA; warps == 0 = TMEM staging (warps per CTA from n_max).
int batch_tmem_warps(int n_max, int Q) {
  const int words = tmem_row_words(n_max, Q <= 254 ? 1 : 2);
  if (words <= 128) return 16;
  if (words <= 256) return 8;
  if (words <= 512) return 4;
  return 0;  // too long for TMEM
}

size_t batch_smem(int n_max, int Q, int warps, int ring, int ns) {
  const int qbytes = Q <= 254 ? 1 : 2;
  if (warps == 0) {
    const int tw = batch_tmem_warps(n_max, Q);
    const size_t need = (size_t)tw * (ring_bytes(ring) + ((size_t)n_max + 2) * sizeof(StepRec));
    return need > kOneCtaPerSmSmem ? need : kOneCtaPerSmSmem;
  }
  return (size_t)warps * ns * ((size_t)32 * staged_row_stride(n_max, qbytes) + ring_bytes(ring));
}

namespace {
template <typename QT, int RING, int NS>
int batch_t(const BatchKernelArgs& a, int warps, int grid, cudaStream_t st, int* occ) {
  const size_t smem = batch_smem(a.n_max, a.Q, warps, RING, warps == 0 ? 1 : NS);
  if (warps == 0) {
    const int tw = batch_tmem_warps(a.n_max, a.Q);
    if (tw == 0) {
      if (occ) *occ = 0;
      return 0;
    }
    auto k = split_batch_tmem_kernel<QT, RING>;
    if (occ) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return (int)e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, tw * 32, smem);
      if (*occ > 1) *occ = 1;  // one TMEM owner per SM
      return (int)e;
    }
    k<<<grid, tw * 32, smem, st>>>(a, 512 / (tw / 4));
    return (int)cudaGetLastError();
  }
  auto k = split_batch_kernel<QT, RING, NS>;
  if (occ) {  // configuration query (never during a stream capture)
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, warps * 32, smem);
  }
  k<<<grid, warps * 32, smem, st>>>(a);
  return (int)cudaGetLastError();
}
template <typename QT, int NS>
int batch_ring(const BatchKernelArgs& a, int warps, int ring, int grid, cudaStream_t st, int* occ) {
  switch (ring) {
    case 8: return batch_t<QT, 8, NS>(a, warps, grid, st, occ);
    case 32: return batch_t<QT, 32, NS>(a, warps, grid, st, occ);
    default: return batch_t<QT, 16, NS>(a, warps, grid, st, occ);
  }
}
}  // namespace

int launch_split_batch(const BatchKernelArgs& a, int warps, int ring, int ns, int grid,
                       cudaStream_t st, int* occ_out) {
  if (ns == 2 && warps > 0)
    return a.Q <= 254 ? batch_ring<uint8_t, 2>(a, warps, ring, grid, st, occ_out)
                      : batch_ring<uint16_t, 2>(a, warps, ring, grid, st, occ_out);
  if (a.Q <= 254) return batch_ring<uint8_t, 1>(a, warps, ring, grid, st, occ_out);
  return batch_ring<uint16_t, 1>(a, warps, ring, grid, st, occ_out);
}

// ---- fused adjoint with TMEM staging

int split_tmem_adj_warps(int n, int Q, int64_t S, int sms) {
  if (n < 1 || S < 1 || sms < 1 || !deque_supported(n, Q)) return 0;
  const int words = tmem_row_words(n, Q <= 254 ? 1 : 2);
  if (words > tmem_cols_per_warp(16)) return 0;
  const int64_t tiles = (S + 31) / 32;
  // 17..24 warps only when they take every tile in one round where 16 need
  // two: a wide round (80 registers a thread) costs more than a 16-warp one,
  // so over several rounds fewer of them did not pay (n = 300 forward: 0.148
  // -> 0.125 ms at 10^5 scenarios, one round; 0.240 -> 0.249 ms at 2 10^5
  // and 0.99 -> 1.10 ms at 10^6, fewest rounds at 21..23 warps)
  const int64_t nw = (tiles + sms - 1) / sms;
  if (nw <= 16 || nw > kTmemMaxWarps || words > tmem_cols_per_warp((int)nw)) return 16;
  return (int)nw;
}

size_t split_tmem_adj_scratch_bytes(int n, int Q, int sms) {
  const int per = Q <= 254 ? 4 : 2;
  return (size_t)sms * kTmemMaxWarps * (size_t)((n + per - 1) / per) * 32 * sizeof(uint32_t);
}

namespace {
template <typename QT>
int launch_adj_t(const SplitDequeArgs& a, int nw, uint32_t* dscratch, int sms,
                 cudaStream_t st) {
  auto k = nw <= 16 ? split_tmem_adj_kernel<QT, 512> : split_tmem_adj_kernel<QT, 32 * kTmemMaxWarps>;
  size_t smem = ((size_t)a.n + 2) * sizeof(StepRec) + cs_bytes(a.n) + (((size_t)(2 * a.n + 1) * 4 + 15) & ~(size_t)15) +
                (size_t)nw * ring_bytes(16);
  if (smem < kOneCtaPerSmSmem) smem = kOneCtaPerSmSmem;  // one TMEM owner per SM
  if (smem > kMaxSmemPerCta) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t tiles = (a.S + 31) / 32;
  const int64_t ctas = (tiles + nw - 1) / nw;
  const int grid = (int)(ctas < sms ? ctas : sms);
  k<<<grid, 32 * nw, smem, st>>>(a, tiles, tmem_cols_per_warp(nw), dscratch);
  return (int)cudaGetLastError();
}
}  // namespace

int launch_split_tmem_adj(const SplitDequeArgs& a, int warps, uint32_t* dscratch, int sms,
                          cudaStream_t st) {
  if (warps < 16 || warps > kTmemMaxWarps || !a.hist || !dscratch) return (int)cudaErrorInvalidValue;
  if (a.Q <= 254) return launch_adj_t<uint8_t>(a, warps, dscratch, sms, st);
  return launch_adj_t<uint16_t>(a, warps, dscratch, sms, st);
}

int deque_max_ctas_per_sm(const DequeConfig& c, bool hist, int pred_dtype,
                          bool want_pred, int* out) {
  SplitDequeArgs a{};
  a.pred_dtype = pred_dtype;
  return dispatch(a, c, out_mode(hist, want_pred), 0, nullptr, out);
}

}  // namespace sdp

// split_deque.cu -- the tuned Split kernel (SDP_ALGO_DEQUE) for sm_103a.
//
// Mapping.  One warp owns a tile of 32 scenarios (one per lane) at a time and
// walks the tour positions i = 1..n in lockstep, so the per-position tour
// record is a warp-uniform broadcast load.  Warps are independent: no CTA
// barrier inside the tile loop, and the grid is persistent (a multiple of the
// SM count times the CTAs that fit per SM).
//
// Staging.  The tile's demand rows are contiguous in HBM (row-major [S, n]);
// the warp reads them with coalesced 16-byte loads and stores them into
// shared memory clamped to Q+1 as uint8 (Q <= 254) or uint16, with a row
// stride whose word count is odd, so the 32 lanes reading the same column of
// 32 rows hit 32 different banks.  While a tile is processed, the next tile of
// the same warp is prefetched into L2 with one bulk (TMA-engine) prefetch.
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
//   - the front is the argmin.
// The deque is a ring of RING entries per lane in shared memory, laid out
// [entry][lane] so every access is bank-conflict free.  A scenario whose
// deque outgrows the ring, or (uint8 staging) whose route would span more
// than 255 customers, is flagged and recomputed by the plain kernel.
//
// Outputs.  The predecessor distance i - pred(i) overwrites, in place, the
// staged demand byte of customer s_i (dead once read), so the tile's
// predecessors are written out afterwards with coalesced row stores.  In the
// fused adjoint the same bytes are backtracked on chip into shared-memory
// route start / end histograms.
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

// Bulk prefetch of [p, p+bytes) into L2 (executed by the TMA engine; p and
// bytes must be multiples of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ StepRec ld_rec(const StepRec* p) {
  int4 v = __ldg(reinterpret_cast<const int4*>(p));
  StepRec r;
  r.col = (uint32_t)v.x;
  r.a = __int_as_float(v.y);
  r.ce = __int_as_float(v.z);
  r.pad = 0u;
  return r;
}

template <typename QT>
__device__ __forceinline__ void put_q(QT* qb, int rs_elems, int r, int c, int v,
                                      int qcap, bool& neg) {
  neg |= v < 0;
  v = min(max(v, 0), qcap);
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

namespace {

// Coalesced 16-byte loads of `rows` contiguous demand rows of n int32 each,
// clamped to [0, Q+1] and stored as narrow rows of rs_elems elements.
template <typename QT>
__device__ __forceinline__ void ingest_tile(const int32_t* src, int rows, int n,
                                            int rs_elems, int qcap, QT* qb, int lane,
                                            bool& neg) {
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
          put_q<QT>(qb, rs_elems, rr, cc, vals[k], qcap, neg);
        }
      }
    }
    for (int64_t f = (nvec << 2) + lane; f < count; f += 32) {
      const int r = (int)(f / n), c = (int)(f - (int64_t)r * n);
      put_q<QT>(qb, rs_elems, r, c, ld_stream_s32(src + f), qcap, neg);
    }
  } else {
    for (int64_t f = lane; f < count; f += 32) {
      const int r = (int)(f / n), c = (int)(f - (int64_t)r * n);
      put_q<QT>(qb, rs_elems, r, c, ld_stream_s32(src + f), qcap, neg);
    }
  }
}

// Warm L2 with `bytes` bytes at p (16-byte aligned interior only).
__device__ __forceinline__ void prefetch_region(const void* p, int64_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pa = (a + 15) & ~(uintptr_t)15;
  int64_t rem = ((bytes - (int64_t)(pa - a)) / 16) * 16;
  for (int64_t o = 0; rem > 0; o += 1 << 20, rem -= 1 << 20)
    prefetch_l2_bulk(reinterpret_cast<const void*>(pa + o), (uint32_t)imin64(rem, 1 << 20));
}

// The DP of one scenario on its staged row (see the file comment).  Leaves
// i - pred(i) in row[col_i]; returns K(n).  first_inf = first position whose
// demand exceeds Q (n+1 if none); bad = the scenario needs the plain path.
template <typename QT, int RING>
__device__ __forceinline__ float dp_row(QT* row, int n, int Q, const StepRec* rec,
                                        float* ring_psi, uint32_t* ring_meta, int lane,
                                        uint32_t& first_inf, bool& bad) {
  const uint32_t maxdelta = sizeof(QT) == 1 ? 255u : 65535u;
  int head = 0, tail = 0;
  int L = 0;
  float K = 0.f, bpsi = 0.f, fpsi = 0.f;
  uint32_t fmeta = 0u;
  StepRec rn = ld_rec(rec);
  int qn = (int)row[rn.col];
  for (int i = 1; i <= n; ++i) {
    const StepRec r = rn;
    const int q = qn;
    if (i < n) rn = ld_rec(rec + i);
    // push p = i-1 after dropping every back entry with a larger psi
    const float psi = __fadd_rn(K, r.a);
    const uint32_t meta = ((uint32_t)L << 16) | (uint32_t)(i - 1);
    while (tail > head && bpsi > psi) {
      --tail;
      if (tail > head) bpsi = ring_psi[((tail - 1) & (RING - 1)) * 32 + lane];
    }
    ring_psi[(tail & (RING - 1)) * 32 + lane] = psi;
    ring_meta[(tail & (RING - 1)) * 32 + lane] = meta;
    ++tail;
    bpsi = psi;
    if (tail - head == 1) { fpsi = psi; fmeta = meta; }
    bad |= (tail - head) > RING;
    // extend the window's right end to customer s_i
    L += q;
    if (q > Q && first_inf > (uint32_t)n) first_inf = (uint32_t)i;
    if (i < n) qn = (int)row[rn.col];
    // drop predecessors whose route s_{p+1..i} exceeds Q
    while (tail - head > 1 && (((uint32_t)L - (fmeta >> 16)) & 0xFFFFu) > (uint32_t)Q) {
      ++head;
      const int h = (head & (RING - 1)) * 32 + lane;
      fpsi = ring_psi[h];
      fmeta = ring_meta[h];
    }
    K = __fadd_rn(fpsi, r.ce);
    const uint32_t delta = (uint32_t)i - (fmeta & 0xFFFFu);
    if (delta > maxdelta && first_inf > (uint32_t)n) bad = true;
    row[r.col] = (QT)delta;
  }
  return K;
}

}  // namespace

template <typename QT, typename PT, int RING, bool HIST>
__global__ void __launch_bounds__(512) split_deque_kernel(SplitDequeArgs a,
                                                          int row_stride,
                                                          int64_t tiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, Q = a.Q;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int rs_elems = row_stride / (int)sizeof(QT);

  // ---- CTA-shared: compact column list (copy-out, backtrack), histograms
  uint16_t* cols_sm = reinterpret_cast<uint16_t*>(smem);
  size_t off = ((size_t)n * 2 + 15) & ~(size_t)15;
  unsigned int* hist_sm = nullptr;
  if (HIST) {
    hist_sm = reinterpret_cast<unsigned int*>(smem + off);
    off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
  }
  const size_t per_warp = (size_t)32 * row_stride + (size_t)RING * 32 * 8;
  unsigned char* wbase = smem + off + per_warp * warp;
  QT* qb = reinterpret_cast<QT*>(wbase);
  float* ring_psi = reinterpret_cast<float*>(wbase + (size_t)32 * row_stride);
  uint32_t* ring_meta = reinterpret_cast<uint32_t*>(ring_psi + RING * 32);

  for (int k = threadIdx.x; k < n; k += blockDim.x) cols_sm[k] = a.cols[k];
  if (HIST)
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x) hist_sm[k] = 0u;
  __syncthreads();

  const double Dn = *a.Dn;
  bool neg = false;
  uint32_t any_inf = 0, any_fb = 0;

  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  for (int64_t tile = (int64_t)blockIdx.x * nwarps + warp; tile < tiles;
       tile += wstride) {
    const int64_t s0 = tile * 32;
    const int rows = (int)imin64(32, a.S - s0);
    ingest_tile<QT>(a.demands + s0 * n, rows, n, rs_elems, Q + 1, qb, lane, neg);
    // warm L2 with this warp's next tile while the DP runs
    if (lane == 0 && tile + wstride < tiles) {
      const int64_t ns0 = (tile + wstride) * 32;
      prefetch_region(a.demands + ns0 * n, imin64(32, a.S - ns0) * n * 4);
    }
    __syncwarp();

    // -------- DP, one scenario per lane
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    if (lane < rows) {
      const float K = dp_row<QT, RING>(qb + lane * rs_elems, n, Q, a.rec, ring_psi,
                                       ring_meta, lane, first_inf, bad);
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (uint32_t)(s0 + lane);
      } else if (a.cost) {
        a.cost[s0 + lane] = first_inf <= (uint32_t)n ? CUDART_INF_F
                                                      : (float)((double)K + Dn);
      }
    }
    const uint32_t fb_mask = __ballot_sync(0xffffffffu, bad);
    const uint32_t inf_mask = __ballot_sync(0xffffffffu, lane < rows && first_inf <= (uint32_t)n);
    any_inf |= inf_mask;
    any_fb |= fb_mask;
    __syncwarp();

    // -------- predecessors: coalesced row stores from the in-place deltas
    if (a.pred) {
      PT* dst0 = reinterpret_cast<PT*>(a.pred) + s0 * n;
      for (int r = 0; r < rows; ++r) {
        const uint32_t fi = __shfl_sync(0xffffffffu, first_inf, r);
        if ((fb_mask >> r) & 1u) continue;
        const QT* row = qb + r * rs_elems;
        PT* dst = dst0 + (int64_t)r * n;
        for (int i = 1 + lane; i <= n; i += 32) {
          const int d = (int)row[cols_sm[i - 1]];
          const int p = (uint32_t)i >= fi ? -1 : i - d;
          dst[i - 1] = (PT)p;
        }
      }
    }
    // -------- fused adjoint: backtrack on chip, count route starts / ends
    if (HIST && lane < rows && !bad && first_inf > (uint32_t)n) {
      const QT* row = qb + lane * rs_elems;
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
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
  if (HIST) {
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * n + 1; k += blockDim.x)
      if (hist_sm[k]) atomicAdd(&a.hist[k], (unsigned long long)hist_sm[k]);
  }
}

// Batched Split: a persistent grid pulls work items (tour, 32-scenario tile)
// from a global counter; items are ordered longest tour first, so the uneven
// tours finish together.  Each warp grabs its next item before working on the
// current one and warms L2 with that item's demand rows.
template <typename QT, int RING>
__global__ void __launch_bounds__(512) split_batch_kernel(BatchKernelArgs a) {
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
    ingest_tile<QT>(a.demands + a.dem_off[b] + s0 * n, rows, n, rs_elems, Q + 1, qb, lane, neg);
    const int64_t next = pop();
    if (lane == 0 && next < items) {
      const int nb = a.order[next / tiles];
      const int64_t ns0 = (next % tiles) * 32;
      const int nn = a.n[nb];
      prefetch_region(a.demands + a.dem_off[nb] + ns0 * nn, imin64(32, a.S - ns0) * nn * 4);
    }
    __syncwarp();
    uint32_t first_inf = (uint32_t)n + 1;
    bool bad = false;
    if (lane < rows) {
      const float K = dp_row<QT, RING>(qb + lane * rs_elems, n, Q, a.rec + a.rec_off[b],
                                       ring_psi, ring_meta, lane, first_inf, bad);
      const int64_t g = (int64_t)b * a.S + s0 + lane;
      if (bad) {
        const uint32_t k = atomicAdd(a.fb_count, 1u);
        a.fb_list[k] = (unsigned long long)g;
      } else {
        a.costs[g] = first_inf <= (uint32_t)n ? CUDART_INF_F
                                               : (float)((double)K + a.Dn[b]);
      }
    }
    any_inf |= __ballot_sync(0xffffffffu, lane < rows && first_inf <= (uint32_t)n);
    any_fb |= __ballot_sync(0xffffffffu, bad);
    __syncwarp();
    item = next;
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
  }
  if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
}

// ------------------------------------------------------------------ host side
bool deque_supported(int n, int Q) { return n >= 1 && n <= 65534 && Q >= 1 && Q <= 32767; }

DequeConfig deque_config(int n, int Q, int warps, int ring, bool hist) {
  DequeConfig c;
  c.warps = warps;
  c.ring = ring;
  c.qbytes = Q <= 254 ? 1 : 2;
  const int rs = staged_row_stride(n, c.qbytes);
  c.row_stride = rs;
  size_t off = ((size_t)n * 2 + 15) & ~(size_t)15;
  if (hist) off += ((size_t)(2 * n + 1) * 4 + 15) & ~(size_t)15;
  c.smem = off + (size_t)warps * ((size_t)32 * rs + (size_t)ring * 32 * 8);
  return c;
}

namespace {
template <typename QT, typename PT, int RING, bool HIST>
int launch_t(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
             int* occ_out) {
  auto k = split_deque_kernel<QT, PT, RING, HIST>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)c.smem);
  if (e != cudaSuccess) return (int)e;
  if (occ_out) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ_out, k, c.warps * 32, c.smem);
    return (int)e;
  }
  const int64_t tiles = (a.S + 31) / 32;
  k<<<grid, c.warps * 32, c.smem, st>>>(a, c.row_stride, tiles);
  return (int)cudaGetLastError();
}

template <typename QT, typename PT, bool HIST>
int by_ring(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
            int* occ) {
  switch (c.ring) {
    case 8: return launch_t<QT, PT, 8, HIST>(a, c, grid, st, occ);
    case 32: return launch_t<QT, PT, 32, HIST>(a, c, grid, st, occ);
    default: return launch_t<QT, PT, 16, HIST>(a, c, grid, st, occ);
  }
}

template <typename QT>
int by_pred(const SplitDequeArgs& a, const DequeConfig& c, bool hist, int grid,
            cudaStream_t st, int* occ) {
  if (hist) return by_ring<QT, int32_t, true>(a, c, grid, st, occ);
  if (a.pred && a.pred_dtype == SDP_PRED_U16)
    return by_ring<QT, uint16_t, false>(a, c, grid, st, occ);
  return by_ring<QT, int32_t, false>(a, c, grid, st, occ);
}

int dispatch(const SplitDequeArgs& a, const DequeConfig& c, int grid, cudaStream_t st,
             int* occ) {
  const bool hist = a.hist != nullptr;
  if (c.qbytes == 1) return by_pred<uint8_t>(a, c, hist, grid, st, occ);
  return by_pred<uint16_t>(a, c, hist, grid, st, occ);
}
}  // namespace

int launch_split_deque(const SplitDequeArgs& a, const DequeConfig& c, int grid,
                       cudaStream_t st) {
  return dispatch(a, c, grid, st, nullptr);
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
  a.hist = hist ? reinterpret_cast<unsigned long long*>(16) : nullptr;
  a.pred = want_pred ? reinterpret_cast<void*>(16) : nullptr;
  a.pred_dtype = pred_dtype;
  return dispatch(a, c, 0, nullptr, out);
}

}  // namespace sdp

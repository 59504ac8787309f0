// split_pipe.cu -- pipelined Split (SDP_ALGO_PIPE, and the batched plans'
// pipelined kernel) for sm_103a.
//
// Why.  A DP lane walks its scenario's positions in tour order, so it needs
// the demand of customer s_i at step i.  Holding a whole row by customer on
// chip for the life of a tile (the DEQUE kernels) caps an SM at 16 tiles
// (TMEM) and 8 (shared memory) at n = 500; a lane step of the deque is a
// short dependent chain that needs more warps than that to keep the
// schedulers busy (measured on the bare step at n = 496, S = 10^6: 16 / 24 /
// 32 / 40 warps per SM gave 1.04 / 0.84 / 0.72 / 0.71 ms).  Here:
//
//   producers (1 issuing + 8 narrowing warps): the issuing warp claims work,
//     sets up slots and feeds TMA bulk copies (cp.async.bulk, two 32 KB
//     stages with full / empty mbarriers -- 48 KB in a batched plan, six of
//     16 KB when its tours are short -- L2 evict-first: every demand is read
//     once) of R contiguous int32 demand rows into shared memory; the
//     narrowing warps narrow them to uint8 (Q <= 254) or uint16 (hard
//     capacity: clamped to [0, Q+1]; soft: kept exactly up to the staging
//     type's range), permute them into tour order and write them to the
//     CTA's ring of tile slots (up to kSlots, 32 rows of `stride` bytes
//     each) in global memory.  The ring of all SMs (about 80 MB at n = 500)
//     stays mostly in L2, so the tour-ordered rows are written and read back
//     largely without a DRAM round trip.  A slot is published through a
//     shared counter (release / acquire) by the narrowing warp that completes
//     the item; its readers are warps of the same CTA.
//   DP warps (23): claim the CTA's items in order from a shared counter, one
//     32-scenario tile per warp, one scenario per lane; each lane reads its
//     tour-ordered row 16 positions at a time (one block ahead, from L2)
//     and runs the deque step below; predecessors go through a per-warp
//     shared-memory transpose and leave as 32-byte row segments (the
//     per-lane stores of one word per row that this replaces took 1.8 ms of a
//     1.0 ms kernel's time at n = 496 through their 32 sector requests each).
//   Work: groups of consecutive tiles of one tour (one tile for a single
//     tour, 4 in a batched plan), claimed from a global counter, longest tour
//     first, so the load balances itself.
//
// DP (Eq. eqdpA in the K-form of sdp_internal.cuh): K(i) = min over the
// capacity window of psi(p) + ce_i, psi(p) = K(p) + a_{p+1}, with the window
// candidates kept in a monotone deque per lane (Algorithm "2D Kernel for
// Splitting" in the linear form of Vidal 2016 for hard capacity): pop from
// the back every entry with a larger psi (an equal psi is older and stays:
// smallest p on ties), push p = i - 1, pop from the front every entry whose
// route p+1..i exceeds Q; the front is the argmin.  An entry is
// (psi bits, L(p) << 16 | p) with the prefix load L taken mod 2^16, and the
// lane keeps Lent = L(i) << 16 | i, so "route p+1..i exceeds Q" is the one
// unsigned compare Lent - entry > (Q << 16 | 0xFFFF): the prefix loads of the
// entries tested differ by at most 2Q + 1 < 2^16 (Q <= 32767) and
// i - p < 2^16.  Without a demand above Q in the tile:
//   - a new psi below the front's (the deque minimum) pops every entry, so
//     the deque restarts at the new entry and the back-pop loop needs no
//     emptiness test (it stops at the front at the latest);
//   - the newest entry (route s_i alone, load q_i <= Q) never pops from the
//     front, so neither loop empties the deque;
//   - the deque holds at most 14 entries every 2 steps (the ring has 16): a
//     lane over that is flagged (its scenario is recomputed by the warp
//     kernel of split_rescue.cu) and its deque restarts at its newest entry,
//     so the ring always holds the deque it describes and both loops end.
//     (At n = 500 the largest deque seen in 64,000 seeded scenarios had 12
//     entries; a seeded n = 1000 tour with Q = 400 reached 16 in 6% of its
//     scenarios, which a test every 4 steps at 12 entries flagged.)
// Tiles with a demand above Q (flagged by the producers) take a checked step
// with emptiness tests, the first infeasible position recorded and an exact
// ring test at every push.  Soft capacity (one tour) runs the same deque with
// the expired entries' running minimum (Lane::step_soft / step_soft_chk).
#include <math_constants.h>

#include "async_copy.cuh"
#include "sdp_internal.cuh"

namespace sdp {

namespace {

constexpr int kDp = 23;                        // DP warps per CTA
constexpr int kNarrow = 8;                     // narrowing warps per CTA (+ one issuing warp)
constexpr int kNarrowThreads = kNarrow * 32;
constexpr int kThreads = (kDp + 1 + kNarrow) * 32;  // 1024 threads: 64 registers each
constexpr int kSlots = 32;                     // tile slots per CTA in the ring, at most
// Producer stages.  A chunk (R whole rows of one tile) costs a fixed round
// of barrier and bookkeeping work besides its bytes, so two 32 KB stages beat
// four of 16 KB and eight of 8 KB with the same bytes in flight (copies and
// narrowing alone, n = 500: 0.60 / 0.82 / 0.97 ms; the batched plan 20.8 ->
// 19.0 ms with the per-item release below).  A batched plan, which keeps no
// records and no predecessor stage in shared memory, takes 48 KB stages
// (whole tiles in one chunk up to n = 384: 18.9 -> 18.5 ms); one tour keeps
// 32 KB (48 KB measured 1.165 -> 1.210 ms at n = 500), and a third stage
// helped neither.
//
// A batched plan whose tours are all short (n <= 128: a whole tile is one
// chunk of 16 KB at most) is bound by the round trip of a stage instead
// (copy, narrowing, barrier, next copy: with two stages a CTA got a tile
// every ~2.9 us on 1025 tours of n = 100), so it takes six 16 KB stages.
constexpr int kMaxNStage = 6;
constexpr int kShortTour = 128;
__host__ __device__ constexpr uint32_t pipe_stage_bytes(bool batched, int nstage) {
  return nstage == 2 ? (batched ? 48u : 32u) * 1024u : 16u * 1024u;
}
// tiles per claimed group: one tour takes them one at a time, so that the
// CTAs' tile counts differ by one at most and every DP warp of the launch
// gets within a tile of the same share (groups of 16 left 208 tiles on most
// CTAs, 9.04 rounds of 23 warps, where the mean is 8.94: 1.204 -> 1.174 ms
// at n = 500, S = 10^6); a batched plan claims 4, since every group may
// change the tour (4096 tours, n 20..1000, S = 4096: groups of 64 / 32 / 16
// / 8 / 4 took 19.07 / 18.73 / 18.55 / 18.47 / 18.40 ms).
constexpr int kGroupOne = 1;
constexpr int kGroupBatch = 4;
__host__ __device__ constexpr int pipe_group(bool batched) { return batched ? kGroupBatch : kGroupOne; }
constexpr int kRing = 16;                      // deque entries per lane
constexpr uint32_t kRingBytes = (uint32_t)kRing * 256u;  // 32 lanes x 8 bytes per entry
constexpr uint32_t kRingMask = (uint32_t)(kRing - 1) << 8;
constexpr uint32_t kOutBytes = 32u * 32u;      // predecessor stage per warp: 32 rows x 32 bytes
constexpr int kColsStride = kPipeMaxN + 8;     // uint16 entries per column table
template <typename QT>
__host__ __device__ constexpr int soft_max() { return sizeof(QT) == 1 ? 255 : 32767; }
constexpr int kCheckEvery = 2;                 // steps between ring tests (lean step)
constexpr uint32_t kMaxAtCheck = 14u;          // entries allowed at a test (+2 pushes <= 16)
static_assert(kMaxAtCheck + kCheckEvery <= (uint32_t)kRing && 16 % kCheckEvery == 0,
              "a test must leave room for the pushes until the next one");

// Stage bookkeeping written by the issuing warp before it arms the stage's
// full barrier (release), read by the narrowing warps after their wait on it
// (acquire).
struct StageMeta {
  int32_t slot, rbase, rows, n;
  int32_t gen;   // tour generation: the narrowing warps reload their columns when it changes
  int32_t stop;  // no more chunks: the narrowing warps leave
  uint32_t item; // item of the chunk
  int32_t pad;
};

__device__ __forceinline__ uint32_t atom_add_acq_rel_shared(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
               : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void mbar_arrive_relaxed(uint32_t bar) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Wait for phase `parity` of an mbarrier, giving up on the abort flag or
// after limit_ns; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_abortable(uint32_t bar, uint32_t parity,
                                                    const uint32_t* abort_flag, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (ld_acquire_shared(abort_flag) || global_ns() - t0 > limit_ns) return false;
  }
}

// ------------------------------------------------------------------ the DP
// One lane's deque (see the file comment).  Ring slots are byte offsets,
// multiples of 256 (32 lanes x 8 bytes), kept unwrapped and masked on use.
struct Lane {
  uint32_t rb;          // shared address of this lane's entry in ring slot 0
  uint32_t head, tail;  // offsets of the front and of the next free slot
  uint32_t Lent;        // L(i) << 16 | i (lean); L(i) << 16 (checked)
  uint32_t fent;        // front entry: L(p) << 16 | p
  float K, fpsi, bpsi;
  bool ovf;             // the deque outgrew the ring: recompute the scenario
  // soft capacity: the best expired entry, c = psi(p) - beta L(p), and its
  // entry; won: the expired candidate is position i's minimum; ovfL: the
  // prefix load passed 2^16, where the entries' L(p) no longer hold it
  float cmin;
  uint32_t cent;
  bool won, ovfL;

  // rings start on 4 KB and a lane's entry is its 8 bytes of a 256-byte
  // slot, so the slot offset and the lane base share no bits: one LOP3
  __device__ __forceinline__ uint32_t at(uint32_t off) const { return rb | (off & kRingMask); }
  __device__ __forceinline__ void init(uint32_t ring, int lane) {
    rb = ring + 8u * (uint32_t)lane;
    head = tail = 0u;
    Lent = fent = 0u;
    K = 0.f;
    fpsi = CUDART_INF_F;  // the first step restarts the deque at p = 0
    bpsi = -CUDART_INF_F;
    ovf = false;
    cmin = CUDART_INF_F;
    cent = 0u;
    won = ovfL = false;
  }
  // position i: demand qh = q_i << 16 and record (a_i, ce_i); no demand
  // above Q in the tile
  __device__ __forceinline__ void step(uint32_t qh, float a, float ce, uint32_t Qc) {
    const float psi = __fadd_rn(K, a);
    const uint32_t ent = Lent;
    Lent += qh + 1u;
    if (psi < fpsi) {  // below the minimum: every entry pops
      tail = head;
      fpsi = psi;
      fent = ent;
      bpsi = -CUDART_INF_F;
    }
    while (bpsi > psi) {
      tail -= 256u;
      bpsi = lds_f32(at(tail - 256u));
    }
    sts_u2(at(tail), __float_as_uint(psi), ent);
    tail += 256u;
    bpsi = psi;
    while (Lent - fent > Qc) {
      head += 256u;
      const uint2 e = lds_u2(at(head));
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
    K = __fadd_rn(fpsi, ce);
  }
  // every kCheckEvery lean steps: more than kMaxAtCheck entries flags the
  // lane and restarts its deque at the newest entry
  __device__ __forceinline__ void check() {
    if (tail - head > kMaxAtCheck * 256u) {
      ovf = true;
      head = tail - 256u;
      const uint2 e = lds_u2(at(head));
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
  }
  // Soft capacity (a route pays beta per unit of load above Q; every split
  // allowed).  An entry leaving from the front joins the expired set, whose
  // best candidate at position i is cmin + beta (L(i) - Q), cmin the least
  // psi(p) - beta L(p) (entries expire in increasing p: "<" keeps the
  // smallest p); an entry leaving from the back is dominated in both regimes.
  // K(i) = min(window minimum, that candidate) + ce_i, ties to the expired
  // entry (the smaller p): the FP32 operations of the DEQUE soft kernel.
  __device__ __forceinline__ void soft_best(float ce, int Q, float beta) {
    float best = fpsi;
    won = false;
    if (cmin < CUDART_INF_F) {
      const float c2 = __fadd_rn(__fmul_rn(beta, (float)((int)(Lent >> 16) - Q)), cmin);
      if (c2 <= best) {
        best = c2;
        won = true;
      }
    }
    K = __fadd_rn(best, ce);
  }
  __device__ __forceinline__ void expire_front(float beta) {
    const float c = __fsub_rn(fpsi, __fmul_rn(beta, (float)(fent >> 16)));
    if (c < cmin) {
      cmin = c;
      cent = fent;
    }
  }
  // lean form: no demand above Q in the tile, so the newest entry stays
  __device__ __forceinline__ void step_soft(uint32_t qh, float a, float ce, uint32_t Qc, int Q,
                                            float beta) {
    const float psi = __fadd_rn(K, a);
    const uint32_t ent = Lent;
    Lent += qh + 1u;
    ovfL |= Lent < ent;
    if (psi < fpsi) {
      tail = head;
      fpsi = psi;
      fent = ent;
      bpsi = -CUDART_INF_F;
    }
    while (bpsi > psi) {
      tail -= 256u;
      bpsi = lds_f32(at(tail - 256u));
    }
    sts_u2(at(tail), __float_as_uint(psi), ent);
    tail += 256u;
    bpsi = psi;
    while (Lent - fent > Qc) {
      expire_front(beta);
      head += 256u;
      const uint2 e = lds_u2(at(head));
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
    soft_best(ce, Q, beta);
  }
  // checked form (Lent = L(i-1) << 16): a demand above Q expires the newest
  // entry too, and an emptied window reads +inf
  __device__ __forceinline__ void step_soft_chk(int i, uint32_t qh, float a, float ce, uint32_t Qc,
                                                int Q, float beta) {
    const float psi = __fadd_rn(K, a);
    const uint32_t ent = Lent | (uint32_t)(i - 1);
    while (bpsi > psi) {
      tail -= 256u;
      bpsi = tail == head ? -CUDART_INF_F : lds_f32(at(tail - 256u));
    }
    if (tail == head) {
      fpsi = psi;
      fent = ent;
    }
    if (tail - head >= kRingBytes) {  // full: flagged, restart at the new entry
      ovf = true;
      head = tail;
      fpsi = psi;
      fent = ent;
    }
    sts_u2(at(tail), __float_as_uint(psi), ent);
    tail += 256u;
    bpsi = psi;
    const uint32_t Lp = Lent;
    Lent += qh;
    ovfL |= Lent < Lp;
    while (head != tail && ((Lent | 0xFFFFu) - fent) > Qc) {
      expire_front(beta);
      head += 256u;
      if (head != tail) {
        const uint2 e = lds_u2(at(head));
        fpsi = __uint_as_float(e.x);
        fent = e.y;
      }
    }
    if (head == tail) {
      fpsi = CUDART_INF_F;
      bpsi = -CUDART_INF_F;
    }
    soft_best(ce, Q, beta);
  }
  // position i of a tile with a demand above Q (Lent = L(i-1) << 16 here)
  __device__ __forceinline__ void step_chk(int i, uint32_t qh, float a, float ce, uint32_t Qc,
                                           uint32_t Qh, int n, uint32_t& first_inf) {
    const float psi = __fadd_rn(K, a);
    const uint32_t ent = Lent | (uint32_t)(i - 1);
    while (bpsi > psi) {
      tail -= 256u;
      bpsi = tail == head ? -CUDART_INF_F : lds_f32(at(tail - 256u));
    }
    if (tail == head) {  // emptied: the new entry becomes the front
      fpsi = psi;
      fent = ent;
    }
    if (tail - head >= kRingBytes) {  // full: flagged, restart at the new entry
      ovf = true;
      head = tail;
      fpsi = psi;
      fent = ent;
    }
    const uint32_t naddr = tail;
    sts_u2(at(tail), __float_as_uint(psi), ent);
    tail += 256u;
    bpsi = psi;
    Lent += qh;
    if (qh > Qh && first_inf > (uint32_t)n) first_inf = (uint32_t)i;
    // the newest entry stays even when q_i > Q (the guard)
    while (((Lent | 0xFFFFu) - fent) > Qc && head != naddr) {
      head += 256u;
      const uint2 e = lds_u2(at(head));
      fpsi = __uint_as_float(e.x);
      fent = e.y;
    }
    K = __fadd_rn(fpsi, ce);
  }
};

// demand of position u (0..15) of a 16-position block (V = sizeof(QT)
// 16-byte vectors), shifted to bits 16..31
template <typename QT>
__device__ __forceinline__ uint32_t q_at(const uint4* c, int u) {
  constexpr int V = (int)sizeof(QT);
  constexpr int PER = 4 / (int)sizeof(QT);
  const int w = u / PER, e = u % PER;
  const uint4 v = w < 4 ? c[0] : c[V - 1];  // selects, no indexed array (u may be dynamic)
  const uint32_t x = (w & 3) == 0 ? v.x : (w & 3) == 1 ? v.y : (w & 3) == 2 ? v.z : v.w;
  if (sizeof(QT) == 1) return __byte_perm(x, 0u, 0x4044u | ((uint32_t)e << 8));
  return e == 0 ? (x << 16) : (x & 0xFFFF0000u);
}

// Tour records (a_i, ce_i) of position k + 1: shared memory (one tour) or
// the plan's records through the read-only path.
struct SmemRec2 {
  uint32_t base;  // shared address of float2 [n]
  __device__ __forceinline__ float2 operator()(int k) const {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(base + 8u * (uint32_t)k));
    return v;
  }
};
struct GlobalRec2 {
  const StepRec* p;
  __device__ __forceinline__ float2 operator()(int k) const {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p + k));
    return make_float2(v.y, v.z);
  }
};

// Predecessors of one warp tile through a [32 rows][8 words] shared stage:
// a 32-byte row segment holds W = 32 / sizeof(PT) positions.  Lane l writes
// word j of its row at l * 8 + (j ^ s(l)), s(l) = 2 ((l >> 2) & 3), and the
// flush reads row r word k at r * 8 + (k ^ s(r)).  The swizzle is even, so
// the word pairs a full flush moves as 8 bytes stay in order; the writes
// meet 2-way bank conflicts (a shared-memory cycle, not an issue slot).
template <typename PT>
struct PredStage {
  uint32_t* st;     // this warp's stage
  PT* tile;         // predecessor rows of the tile
  int n, rows, lane;
  bool pairs;       // uint16: every row segment starts on 4 bytes (n even, aligned base)
  bool wide;        // every row segment starts on 8 bytes: full flushes store 8 bytes a lane
  uint32_t pend;    // uint16: the even position of the word being packed (its low half is used)
  static constexpr int W = 32 / (int)sizeof(PT);
  __device__ __forceinline__ void put(int pos, uint32_t p) {  // pos = (i - 1) % W
    const int sw = ((lane >> 2) & 3) << 1;  // even: word pairs stay in order
    if (sizeof(PT) == 2) {
      if ((pos & 1) == 0) {
        pend = p;
      } else {
        st[lane * 8 + ((pos >> 1) ^ sw)] = __byte_perm(pend, p, 0x5410);
      }
    } else {
      st[lane * 8 + (pos ^ sw)] = p;
    }
  }
  // positions i0 .. i0 + cnt - 1 (1-based) of every row
  __device__ __forceinline__ void flush(int i0, int cnt) {
    if (sizeof(PT) == 2 && (cnt & 1)) st[lane * 8 + ((cnt >> 1) ^ (((lane >> 2) & 3) << 1))] = pend;
    __syncwarp();
    constexpr int PER = 4 / (int)sizeof(PT);
    if (wide && cnt == W) {
      // lane: word pair k2 (words 2 k2, 2 k2 + 1) of row 8 m + lane / 4; the
      // pair sits at (2 k2 ^ s) & ~1, swapped when the row's swizzle s is odd
      const int k2 = lane & 3;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int r = 8 * m + (lane >> 2);
        const int sz = ((r >> 2) & 3) << 1;
        const uint2 v = *reinterpret_cast<const uint2*>(st + r * 8 + (2 * k2 ^ sz));
        if (r < rows) {
          PT* dst = tile + (int64_t)r * n + (i0 - 1) + 2 * k2 * PER;
          *reinterpret_cast<uint2*>(dst) = v;
        }
      }
      __syncwarp();
      return;
    }
    const int k = lane & 7;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int r = 4 * m + (lane >> 3);
      const uint32_t v = st[r * 8 + (k ^ ((m & 3) << 1))];
      if (r < rows && k * PER < cnt) {
        PT* dst = tile + (int64_t)r * n + (i0 - 1) + k * PER;
        if (sizeof(PT) == 4) {
          *reinterpret_cast<uint32_t*>(dst) = v;
        } else if (pairs && k * 2 + 1 < cnt) {
          *reinterpret_cast<uint32_t*>(dst) = v;
        } else {
          dst[0] = (PT)(v & 0xFFFFu);
          if (k * 2 + 1 < cnt) dst[1] = (PT)(v >> 16);
        }
      }
    }
    __syncwarp();
  }
};

// One 32-scenario tile: lane l runs scenario s0 + l over positions 1..n from
// its tour-ordered row.  CHECK: the tile has a demand above Q.  SOFT: soft
// capacity with penalty beta per unit of route load above Q.
template <typename QT, typename PT, bool PRED, bool CHECK, bool SOFT, typename REC>
__device__ __forceinline__ void pipe_tile(int n, int Q, float beta, const unsigned char* qrow,
                                          uint32_t ring, const REC rec, int lane, PredStage<PT>& ps,
                                          float* K_out, uint32_t* first_inf_out, bool* bad) {
  constexpr int E = 16;                    // positions per block
  constexpr int V = (int)sizeof(QT);       // 16-byte vectors per block
  constexpr int W = PredStage<PT>::W;      // positions per predecessor flush (16 % W == 0)
  const uint32_t Qh = (uint32_t)Q << 16, Qc = Qh | 0xFFFFu;
  Lane st;
  st.init(ring, lane);
  uint32_t first_inf = (uint32_t)n + 1u;
  const int nblk = n / E;                  // whole blocks
  const int last = (n + E - 1) / E - 1;    // last block holding a position
  const uint4* src = reinterpret_cast<const uint4*>(qrow);
  uint4 c[V];
#pragma unroll
  for (int v = 0; v < V; ++v) c[v] = ld_cg_v4(src + v);
  auto pred_of = [&](int i) -> uint32_t {
    if (!SOFT && CHECK && (uint32_t)i >= first_inf) return 0xFFFFFFFFu;
    const uint32_t e = (SOFT && st.won) ? st.cent : st.fent;
    return sizeof(PT) == 2 ? e : (e & 0xFFFFu);
  };
  // position i; test: the lean step's ring test is due
  auto do_step = [&](int i, uint32_t qh, float2 r, bool test) {
    if (SOFT) {
      if (CHECK) {
        st.step_soft_chk(i, qh, r.x, r.y, Qc, Q, beta);
      } else {
        st.step_soft(qh, r.x, r.y, Qc, Q, beta);
        if (test) st.check();
      }
    } else if (CHECK) {
      st.step_chk(i, qh, r.x, r.y, Qc, Qh, n, first_inf);
    } else {
      st.step(qh, r.x, r.y, Qc);
      if (test) st.check();
    }
  };
  for (int b = 0; b < nblk; ++b) {
    const int bn = min(b + 1, last);
    uint4 nx[V];
#pragma unroll
    for (int v = 0; v < V; ++v) nx[v] = ld_cg_v4(src + V * bn + v);
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int i = b * E + u + 1;
      const float2 r = rec(i - 1);
      const uint32_t qh = q_at<QT>(c, u);
      do_step(i, qh, r, u % kCheckEvery == kCheckEvery - 1);
      if (PRED) {
        ps.put(u % W, pred_of(i));
        if (u % W == W - 1) ps.flush(i - W + 1, W);
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = nx[v];
  }
  // ragged tail (fewer than E positions) from the block loaded last
  const int i1 = nblk * E + 1;
  for (int i = i1; i <= n; ++i) {
    const int u = i - i1;
    const float2 r = rec(i - 1);
    const uint32_t qh = q_at<QT>(c, u);
    do_step(i, qh, r, true);
    if (PRED) {
      ps.put(u % W, pred_of(i));
      if (u % W == W - 1 || i == n) ps.flush(i - u % W, u % W + 1);
    }
  }
  *K_out = st.K;
  *first_inf_out = first_inf;
  *bad = st.ovf || (SOFT && st.ovfL);
}

// ------------------------------------------------------------------ kernel
template <typename QT, typename PT, bool PRED, bool BATCH, bool SOFT, int NST>
__global__ void __launch_bounds__(kThreads, 1) split_pipe_kernel(PipeArgs a) {
  constexpr int kNStage = NST;  // producer stages of this launch
  static_assert(NST >= 2 && NST <= kMaxNStage, "stage count");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxNStage], empty_bar[kMaxNStage];
  __shared__ StageMeta smeta[kMaxNStage];
  __shared__ uint32_t slot_ready[kSlots], slot_free[kSlots], slot_inf[kSlots];
  __shared__ uint32_t slot_fb[kSlots];  // soft: rows with a demand the staging type cannot hold
  __shared__ uint32_t item_cnt[kSlots], item_need[kSlots];
  __shared__ int32_t slot_b[kSlots];
  __shared__ int64_t slot_s0[kSlots];
  __shared__ uint32_t next_item, final_count, abort_flag;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int Q = a.Q;
  const int64_t S = a.S;
  // shared: stages | DP rings | predecessor stages | (one tour) records | columns
  constexpr uint32_t kStage = pipe_stage_bytes(BATCH, NST);  // bytes per producer stage
  const uint32_t rings = (smem_u32(smem) + kNStage * kStage + kRingBytes - 1) & ~(kRingBytes - 1);
  const size_t rings_off = rings - smem_u32(smem);  // (the smem size holds kRingBytes of slack)
  uint32_t* ostage = reinterpret_cast<uint32_t*>(smem + rings_off + (size_t)kDp * kRingBytes);
  unsigned char* tail_sm = smem + rings_off + (size_t)kDp * kRingBytes +
                           (PRED ? (size_t)kDp * kOutBytes : 0);
  float2* rec2 = reinterpret_cast<float2*>(tail_sm);
  // the tour's columns; a batched plan keeps two tables, by tour generation
  // parity, so that the issuer can write the next tour's while chunks of the
  // current one are narrowed
  uint16_t* cols0 = reinterpret_cast<uint16_t*>(tail_sm + (BATCH ? 0 : (size_t)a.n1 * sizeof(float2)));
  auto cols_of = [&](int g) -> uint16_t* { return cols0 + (BATCH ? (g & 1) * kColsStride : 0); };
  // stage k: full (the issuer's expect_tx + the bulk copy) and empty (one
  // arrival per narrowing warp) barriers
  const uint32_t full0 = smem_u32(&full_bar[0]), empty0 = smem_u32(&empty_bar[0]);
  if (threadIdx.x == 0) {
    for (int k = 0; k < kNStage; ++k) {
      mbar_init(full0 + 8u * k, 1);
      mbar_init(empty0 + 8u * k, kNarrow);
    }
    mbar_fence_init();
    next_item = 0u;
    final_count = 0xFFFFFFFFu;
    abort_flag = 0u;
  }
  if (threadIdx.x < kSlots) {
    slot_ready[threadIdx.x] = 0u;
    slot_free[threadIdx.x] = 0u;
  }
  if (!BATCH) {
    for (int k = threadIdx.x; k < a.n1; k += blockDim.x) {
      const StepRec r = a.rec[k];
      rec2[k] = make_float2(r.a, r.ce);
    }
  }
  __syncthreads();
  const uint32_t nslot = (uint32_t)a.nslot;  // this launch's slots per CTA (<= kSlots)
  unsigned char* qslots = a.qt + (int64_t)blockIdx.x * nslot * 32 * a.stride;
  const int64_t tpt = (S + 31) / 32;                 // tiles per tour
  constexpr int kGroup = pipe_group(BATCH);
  const int64_t gpt = (tpt + kGroup - 1) / kGroup;   // groups per tour
  const int64_t groups = gpt * a.B;

  constexpr int PER = 4 / (int)sizeof(QT);  // demands per 32-bit slot word
  constexpr int kSoftMax = soft_max<QT>();
  auto full_of = [&](int64_t x) -> uint32_t { return full0 + 8u * (uint32_t)(x % kNStage); };
  auto empty_of = [&](int64_t x) -> uint32_t { return empty0 + 8u * (uint32_t)(x % kNStage); };
  auto par_of = [&](int64_t x) -> uint32_t { return (uint32_t)(x / kNStage) & 1u; };

  if (warp == kDp) {
    // ------------------------------------------------------------ issuer
    // Claims groups, sets up each item's slot, and feeds chunk x (R rows of
    // one tile) into stage x % kNStage once chunk x - kNStage has been
    // narrowed.  Lane 0 does the single-thread work; the warp loads columns.
    const uint64_t pol = l2_evict_first_policy();
    int cur_b = -1, n = 0, R = 32, subs = 1, gen = 0;
    int64_t gen_x0e = -1, gen_x0o = -1;  // first chunk of the latest even / odd generation
    uint32_t li = 0;  // items set up by this CTA
    int64_t x = 0;    // chunks issued
    bool failed = false;
    // chunk y narrowed (its stage free again), or give up
    auto wait_done = [&](int64_t y) -> bool {
      return y < 0 || mbar_wait_abortable(empty_of(y), par_of(y), &abort_flag, a.wait_ns);
    };
    while (!failed) {
      int64_t gid = 0;
      if (lane == 0) gid = (int64_t)atomicAdd(a.counter, 1ull);
      gid = __shfl_sync(0xffffffffu, gid, 0);
      if (gid >= groups) break;
      const int b = BATCH ? a.order[gid / gpt] : 0;
      const int64_t t0 = (gid % gpt) * kGroup;
      const int m = (int)imin64(kGroup, tpt - t0);  // items in the group
      if (b != cur_b) {
        // a new tour: its table is the one of two generations ago, which
        // the narrowing warps read at that generation's first chunk (chunks
        // are narrowed in order, so that chunk done is enough)
        ++gen;
        const int64_t y0 = (gen & 1) ? gen_x0o : gen_x0e;
        const bool ok = y0 < x - kNStage || wait_done(y0);
        if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
        if (gen & 1) gen_x0o = x; else gen_x0e = x;
        cur_b = b;
        n = BATCH ? a.n[b] : a.n1;
        const int wqp = ((n + PER - 1) / PER) * PER;
        const StepRec* rec = a.rec + (BATCH ? a.rec_off[b] : 0);
        uint16_t* cols = cols_of(gen);
        for (int k = lane; k < wqp; k += 32)
          cols[k] = k < n ? (BATCH ? (uint16_t)rec[k].col : a.cols[k]) : (uint16_t)0;
        R = 32;
        while ((uint32_t)R * (uint32_t)n * 4u > kStage) R >>= 1;
        subs = 32 / R;
        __syncwarp();
      }
      const int32_t* dem = a.demands + (BATCH ? a.dem_off[b] : 0);
      for (int j = 0; j < m && !failed; ++j) {
        const uint32_t item = li + (uint32_t)j;
        const uint32_t slot = item % nslot;
        const int64_t s0 = (t0 + j) * 32;
        bool ok = true;
        if (lane == 0) {
          // the slot's previous item (item - nslot) must be finished
          if (item >= nslot) {
            const uint32_t need = item - nslot + 1;
            const uint64_t tw = global_ns();
            while (ld_acquire_shared(&slot_free[slot]) < need) {
              if (ld_acquire_shared(&abort_flag) || global_ns() - tw > a.wait_ns) {
                ok = false;
                break;
              }
              __nanosleep(256);
            }
          }
          slot_inf[slot] = 0u;
          slot_fb[slot] = 0u;
          slot_b[slot] = b;
          slot_s0[slot] = s0;
          item_cnt[slot] = 0u;
          item_need[slot] = (uint32_t)kNarrow;
        }
        if (!__shfl_sync(0xffffffffu, (int)ok, 0)) { failed = true; break; }
        for (int q = 0; q < subs; ++q) {
          const int64_t r0 = s0 + (int64_t)q * R;
          const int rows = r0 >= S ? 0 : (int)imin64(R, S - r0);
          const bool okw = wait_done(x - kNStage);
          if (!__all_sync(0xffffffffu, okw)) { failed = true; break; }
          if (lane == 0) {
            const int st = (int)(x % kNStage);
            int32_t* sq = reinterpret_cast<int32_t*>(smem + (size_t)st * kStage);
            const uint32_t bytes = ((uint32_t)rows * (uint32_t)n * 4u) & ~15u;
            // the last few demands of a ragged last chunk (not a whole 16 bytes)
            for (int e = (int)(bytes >> 2); e < rows * n; ++e) sq[e] = __ldg(dem + r0 * n + e);
            StageMeta& mt = smeta[st];
            mt.slot = (int32_t)slot;
            mt.rbase = q * R;
            mt.rows = rows;
            mt.n = n;
            mt.gen = gen;
            mt.stop = 0;
            mt.item = item;
            fence_proxy_async();  // the narrowing warps' reads of the stage come first
            mbar_arrive_tx(full_of(x), bytes);
            if (bytes) bulk_g2s_hint(smem_u32(sq), dem + r0 * n, bytes, full_of(x), pol);
          }
          ++x;
        }
      }
      if (!failed) li += (uint32_t)m;
    }
    if (!failed) {
      // a stop marker in the next stage, once it is free
      const bool ok = wait_done(x - kNStage);
      if (!__all_sync(0xffffffffu, ok)) {
        failed = true;
      } else if (lane == 0) {
        StageMeta& mt = smeta[x % kNStage];
        mt.stop = 1;
        mbar_arrive_tx(full_of(x), 0u);
        st_release_shared(&final_count, li);
      }
    }
    if (failed && lane == 0) {
      atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
      st_release_shared(&abort_flag, 1u);
      // let copies still in flight land (again with a time limit) before
      // shared memory goes
      for (int64_t y = x - kNStage < 0 ? 0 : x - kNStage; y < x; ++y) mbar_wait(full_of(y), par_of(y));
    }
    return;
  }

  if (warp > kDp) {
    // ---------------------------------------------------------- narrowing
    // Chunk x: wait for its stage, narrow + permute its rows into the slot
    // (rows past S become zero demands: their lanes run on them, outputs
    // dropped), count it toward the item (the warp completing the item
    // publishes it), free the stage.  Thread t owns words k = kw0 + 128 j of
    // the rows rfirst, rfirst + rstep, ... (the mapping is chosen per tour
    // below), their columns in registers per tour (one word per thread for
    // rows of up to 512 bytes: the slowest thread sets the pace of the
    // stage).
    const int t = (int)threadIdx.x - (kDp + 1) * 32;
    constexpr int kHalf = kNarrowThreads / 2;                       // 128
    constexpr int kWordsMax = kPipeMaxN * (int)sizeof(QT) / 4;      // words per row at most
    constexpr int kWords = (kWordsMax + kHalf - 1) / kHalf;         // words per thread
    const int kw = t % kHalf, rpar = t / kHalf;
    const int sw = (int)(a.stride / 4);  // words per slot row
    uint32_t wcol[kWords][PER];          // byte offset in a stage row of each position
    uint32_t wmask[kWords];              // the word's bits of positions below n
    int cached_gen = -1, n = 0, wq = 0, R = 0;
    int kw0 = kw, rfirst = rpar, rstep = 2;  // this thread's first word, first row and row step
    int mn_all = 0;
    for (int64_t x = 0;; ++x) {
      if (!mbar_wait_abortable(full_of(x), par_of(x), &abort_flag, a.wait_ns)) {
        if (lane == 0) st_release_shared(&abort_flag, 1u);
        break;
      }
      const int st = (int)(x % kNStage);
      const StageMeta mt = smeta[st];
      if (mt.stop) break;
      if (mt.gen != cached_gen) {
        cached_gen = mt.gen;
        n = mt.n;
        wq = (n + PER - 1) / PER;
        R = 32;  // rows per chunk, as the issuer chose them
        while ((uint32_t)R * (uint32_t)n * 4u > kStage) R >>= 1;
        // rows short enough for three or more groups: the kNarrowThreads
        // threads form G = kNarrowThreads / wq groups of wq, group g taking
        // rows g, g + G, ..., so that most threads have a word to narrow
        // (n = 100: 250 of 256, n = 300: 225 instead of 150); longer rows: a
        // thread per word position of its parity's rows (n = 500: 250, and
        // each warp stores 32 words of one row).  A thread keeps one word's
        // columns either way.
        if (kNarrowThreads / wq >= 3) {
          const int G = kNarrowThreads / wq;
          kw0 = t < G * wq ? t % wq : wq;
          rfirst = t < G * wq ? t / wq : 0;
          rstep = G;
        } else {
          kw0 = kw;
          rfirst = rpar;
          rstep = 2;
        }
#pragma unroll
        for (int j = 0; j < kWords; ++j) {
          // a position past n reads the word's first column again (same
          // value: the range test is unchanged) and is masked off after
          // packing
          const int k = kw0 + kHalf * j;
          const uint16_t* cols = cols_of(cached_gen);
          const uint32_t c0 = k < wq ? (uint32_t)cols[PER * k] * 4u : 0u;
          wmask[j] = 0u;
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const bool v = k < wq && PER * k + e < n;
            wcol[j][e] = v ? (uint32_t)cols[PER * k + e] * 4u : c0;
            wmask[j] |= v ? ((sizeof(QT) == 1 ? 0xFFu : 0xFFFFu) << (e * 8 * (int)sizeof(QT))) : 0u;
          }
        }
      }
      const uint32_t slot = (uint32_t)mt.slot;
      const int rows = mt.rows;
      const uint32_t sq_b = smem_u32(smem) + (uint32_t)st * kStage;
      uint32_t* out = reinterpret_cast<uint32_t*>(qslots + ((int64_t)slot * 32 + mt.rbase) * a.stride);
#pragma unroll
      for (int j = 0; j < kWords; ++j) {
        const int k = kw0 + kHalf * j;
        if (k >= wq) break;
        const int r0 = rfirst;
        uint32_t rb = sq_b + (uint32_t)(r0 * n) * 4u;  // stage row r0
        uint32_t* o = out + (int64_t)r0 * sw + k;
        int r = r0;
        for (; r < rows; r += rstep, rb += 4u * (uint32_t)rstep * (uint32_t)n, o += rstep * sw) {
          int v[PER];
#pragma unroll
          for (int e = 0; e < PER; ++e)
            asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v[e]) : "r"(rb + wcol[j][e]));
          uint32_t mx = (uint32_t)v[0];
#pragma unroll
          for (int e = 1; e < PER; ++e) mx = max(mx, (uint32_t)v[e]);
          uint32_t word;
          if (mx <= (uint32_t)Q) {
            word = sizeof(QT) == 1
                       ? __byte_perm(__byte_perm(v[0], v[1 % PER], 0x0040),
                                     __byte_perm(v[2 % PER], v[3 % PER], 0x0040), 0x5410)
                       : __byte_perm(v[0], v[1 % PER], 0x5410);
          } else {
            // a demand above Q or below 0.  Hard capacity: clamp to
            // [0, Q+1] (the tile takes the checked step, the scenario is
            // infeasible).  Soft: kept exactly for the checked step up to
            // kSoftMax (so that Q + q < 2^16 in the front test); beyond it
            // the scenario goes to the plain kernel.
            bool inf = false, big = false;
            word = 0u;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
              inf |= v[e] > Q;
              mn_all = min(mn_all, v[e]);
              big |= SOFT && v[e] > kSoftMax;
              word |= (uint32_t)min(max(v[e], 0), SOFT ? kSoftMax : Q + 1) << (e * 8 * (int)sizeof(QT));
            }
            if (inf) atomicOr(&slot_inf[slot], 1u << (mt.rbase + r));
            if (big) atomicOr(&slot_fb[slot], 1u << (mt.rbase + r));
          }
          *o = word & wmask[j];
        }
        for (; r < R; r += rstep, o += rstep * sw) *o = 0u;  // rows past S
      }
      __syncwarp();
      if (lane == 0) {
        // The stage is free once every lane's shared reads of it are done:
        // their values fed the ring stores above, and the warp has
        // converged, so a relaxed arrival (which waits for no store) does.
        // The item is counted once per warp, after its last chunk, with a
        // release that covers the warp's stores of every chunk of the item.
        // (a.stall: fault injection for tests -- nothing is published, and
        // the DP warps' waits run out after a.wait_ns)
        mbar_arrive_relaxed(empty_of(x));
        if (mt.rbase + R >= 32 &&
            atom_add_acq_rel_shared(&item_cnt[slot], 1u) + 1u == item_need[slot] && !a.stall)
          st_release_shared(&slot_ready[slot], mt.item + 1u);
      }
    }
    if (mn_all < 0) atomicOr(a.status, SDP_FLAG_NEG_INPUT);
    return;
  }

  // ------------------------------------------------------------------ DP warps
  const uint32_t ring = rings + kRingBytes * (uint32_t)warp;
  PredStage<PT> ps{};
  ps.st = ostage + warp * (kOutBytes / 4);
  ps.lane = lane;
  uint32_t any_inf = 0, any_fb = 0;
  bool timed_out = false;
  for (;;) {
    uint32_t li = 0;
    if (lane == 0) li = atomicAdd(&next_item, 1u);
    li = __shfl_sync(0xffffffffu, li, 0);
    const uint32_t slot = li % nslot;
    // wait until item li is published, or the producers are done
    bool have = ld_acquire_shared(&slot_ready[slot]) > li;
    if (!have) {
      const uint64_t tw = global_ns();
      while (true) {
        if (ld_acquire_shared(&slot_ready[slot]) > li) {
          have = true;
          break;
        }
        if (ld_acquire_shared(&final_count) <= li) break;
        if (ld_acquire_shared(&abort_flag)) break;
        if (global_ns() - tw > a.wait_ns) {
          timed_out = true;
          st_release_shared(&abort_flag, 1u);  // producers and the other DP warps stop too
          break;
        }
        __nanosleep(512);  // few polls: a waiting warp leaves the issue slots to the others
      }
    }
    if (!__all_sync(0xffffffffu, have)) break;
    const int b = slot_b[slot];
    const int64_t s0 = slot_s0[slot];
    const uint32_t tf = slot_inf[slot];
    const uint32_t tfb = SOFT ? slot_fb[slot] : 0u;
    const int n = BATCH ? a.n[b] : a.n1;
    const int rows = (int)imin64(32, S - s0);
    const bool live = lane < rows;
    const unsigned char* qrow = qslots + ((int64_t)slot * 32 + lane) * a.stride;
    if (PRED) {
      ps.tile = reinterpret_cast<PT*>(a.pred) + s0 * n;
      ps.n = n;
      ps.rows = rows;
      ps.pairs = sizeof(PT) == 4 || ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.pred) & 3) == 0);
      ps.wide = (n % (8 / (int)sizeof(PT))) == 0 && (reinterpret_cast<uintptr_t>(a.pred) & 7) == 0;
    }
    float K;
    uint32_t first_inf;
    bool bad;
    if (BATCH) {
      const GlobalRec2 rec{a.rec + a.rec_off[b]};
      if (tf)
        pipe_tile<QT, PT, PRED, true, false>(n, Q, 0.f, qrow, ring, rec, lane, ps, &K, &first_inf, &bad);
      else
        pipe_tile<QT, PT, PRED, false, false>(n, Q, 0.f, qrow, ring, rec, lane, ps, &K, &first_inf, &bad);
    } else {
      const SmemRec2 rec{smem_u32(rec2)};
      if (tf)
        pipe_tile<QT, PT, PRED, true, SOFT>(n, Q, a.beta, qrow, ring, rec, lane, ps, &K, &first_inf, &bad);
      else
        pipe_tile<QT, PT, PRED, false, SOFT>(n, Q, a.beta, qrow, ring, rec, lane, ps, &K, &first_inf, &bad);
    }
    __syncwarp();  // every lane is done with the slot
    if (lane == 0) st_release_shared(&slot_free[slot], li + 1);
    bad = (bad || ((tfb >> lane) & 1u)) && live;
    if (live) {
      const int64_t g = BATCH ? (int64_t)b * S + s0 + lane : s0 + lane;
      if (bad) {
        const uint32_t f = atomicAdd(a.fb_count, 1u);
        if (BATCH)
          a.fb_list[f] = (unsigned long long)g;
        else
          a.fb_list1[f] = (uint32_t)g;
      } else {
        a.cost[g] = first_inf <= (uint32_t)n ? CUDART_INF_F : (float)((double)K + a.Dn[b]);
      }
    }
    if (!SOFT) any_inf |= tf;
    any_fb |= __ballot_sync(0xffffffffu, bad);
  }
  if (lane == 0) {
    if (any_inf) atomicOr(a.status, SDP_FLAG_INFEASIBLE);
    if (any_fb) atomicOr(a.status, SDP_FLAG_FALLBACK);
    if (timed_out) atomicOr(a.status, SDP_FLAG_DEVICE_CHECK);
  }
}

int pipe_nstage(const PipeArgs& a) { return a.batched && a.n_max <= kShortTour ? kMaxNStage : 2; }

size_t pipe_smem(const PipeArgs& a, bool pred) {
  const int n = a.batched ? kPipeMaxN : a.n1;
  const int ns = pipe_nstage(a);
  return (size_t)ns * pipe_stage_bytes(a.batched != 0, ns) + (size_t)(kDp + 1) * kRingBytes + (pred ? (size_t)kDp * kOutBytes : 0) +
         (a.batched ? 0 : (size_t)n * sizeof(float2)) +
         (a.batched ? 2 * (size_t)kColsStride : (size_t)n + 8) * sizeof(uint16_t);
}

template <typename QT, typename PT, bool PRED, bool BATCH, bool SOFT = false, int NST = 2>
int launch_k(const PipeArgs& a, cudaStream_t st) {
  auto k = split_pipe_kernel<QT, PT, PRED, BATCH, SOFT, NST>;
  const size_t smem = pipe_smem(a, PRED);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k<<<pipe_grid(a.S, a.B, BATCH), kThreads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename QT>
int launch_q(const PipeArgs& a, cudaStream_t st) {
  if (a.batched)
    return pipe_nstage(a) == kMaxNStage ? launch_k<QT, uint16_t, false, true, false, kMaxNStage>(a, st)
                                        : launch_k<QT, uint16_t, false, true>(a, st);
  if (a.soft) {  // one tour only
    if (!a.pred) return launch_k<QT, uint16_t, false, false, true>(a, st);
    if (a.pred_dtype == SDP_PRED_U16) return launch_k<QT, uint16_t, true, false, true>(a, st);
    return launch_k<QT, int32_t, true, false, true>(a, st);
  }
  if (!a.pred) return launch_k<QT, uint16_t, false, false>(a, st);
  if (a.pred_dtype == SDP_PRED_U16) return launch_k<QT, uint16_t, true, false>(a, st);
  return launch_k<QT, int32_t, true, false>(a, st);
}

}  // namespace

bool pipe_supported(int n, int Q) { return n >= 1 && n <= kPipeMaxN && Q >= 1 && Q <= 32767; }

int pipe_grid(int64_t S, int B, bool batched) {
  const int g = pipe_group(batched);
  const int64_t groups = (int64_t)B * ((((S + 31) / 32) + g - 1) / g);
  return (int)imin64(num_sms(), groups < 1 ? 1 : groups);
}

// slots per CTA: twice a CTA's share of the tiles (a small launch spread over
// many CTAs needs few), 2 to kSlots
int pipe_slots(int64_t S, int B, bool batched) {
  const int grid = pipe_grid(S, B, batched);
  const int64_t items = (int64_t)B * ((S + 31) / 32);
  const int64_t per = (items + grid - 1) / grid;
  return (int)imin64(kSlots, per < 1 ? 2 : 2 * per);
}

size_t pipe_ring_bytes(int n_max, int Q, int64_t S, int B, bool batched) {
  return (size_t)pipe_grid(S, B, batched) * (size_t)pipe_slots(S, B, batched) * 32 *
         (size_t)pipe_row_stride(n_max, Q);
}

int launch_split_pipe(const PipeArgs& a0, cudaStream_t st) {
  PipeArgs a = a0;
  if (a.wait_ns == 0) a.wait_ns = kWaitLimitNs;
  a.nslot = pipe_slots(a.S, a.B, a.batched != 0);
  return a.Q <= 254 ? launch_q<uint8_t>(a, st) : launch_q<uint16_t>(a, st);
}

}  // namespace sdp

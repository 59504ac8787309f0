"""The PIPE kernel's narrowing map, checked on the CPU for every tour length.

In split_pipe.cu each of the 256 narrowing threads writes 4-byte words of a
chunk of tour-ordered rows into a slot of the ring: rows of at most 85 words
are split into G = 256 // words groups (thread t: word t % words of rows
t // words, + G, + 2G, ...), longer rows give each thread the word
positions kw + 128 j of the rows of its parity (t // 128, stride 2); rows
past S are written as zeros on the same stride.  This model restates that
index arithmetic and checks, for n = 1..1024, uint8 and uint16 rows, every
stage size and every chunk height, that each (row, word) of a chunk is
written exactly once, that every stage read stays inside the chunk's rows
and every store inside its slot row.  The source lines the model restates
are asserted to be present, so a change to the kernel's map fails here
until the model follows it."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2602_05179_gb300", "csrc", "split_pipe.cu")
INTERNAL = os.path.join(ROOT, "paper_2602_05179_gb300", "csrc", "sdp_internal.cuh")

NARROW_THREADS, HALF, PIPE_MAX_N = 256, 128, 1024
STAGES = (16 * 1024, 32 * 1024, 48 * 1024)   # pipe_stage_bytes: six 16 KB, or two of 32 / 48 KB


def test_model_follows_the_kernel_source():
    src = open(SRC).read()
    for line in ("constexpr int kNarrow = 8;",
                 "constexpr int kNarrowThreads = kNarrow * 32;",
                 "constexpr int kHalf = kNarrowThreads / 2;",
                 "const int kw = t % kHalf, rpar = t / kHalf;",
                 "if (kNarrowThreads / wq >= 3) {",
                 "const int G = kNarrowThreads / wq;",
                 "kw0 = t < G * wq ? t % wq : wq;",
                 "rfirst = t < G * wq ? t / wq : 0;",
                 "rstep = G;",
                 "kw0 = kw;",
                 "rfirst = rpar;",
                 "rstep = 2;",
                 "const int k = kw0 + kHalf * j;",
                 "if (k >= wq) break;",
                 "for (; r < rows; r += rstep,",
                 "for (; r < R; r += rstep, o += rstep * sw) *o = 0u;",
                 "return nstage == 2 ? (batched ? 48u : 32u) * 1024u : 16u * 1024u;"):
        assert line in src, line
    assert src.count("while ((uint32_t)R * (uint32_t)n * 4u > kStage) R >>= 1;") == 2
    assert "constexpr int kPipeMaxN = 1024;" in open(INTERNAL).read()


def _chunk_rows(n, stage):
    R = 32
    while R * n * 4 > stage:
        R >>= 1
    return R


def _writes(n, qbytes, rows, R):
    """(row, word) of every store the 256 threads make for one chunk.  A
    store of word k at a row below `rows` reads stage row r at the columns
    of positions per*k .. per*k + per - 1 (those past n read position per*k
    again): all below n, so inside the chunk when R*n*4 fits the stage."""
    per = 4 // qbytes
    wq = (n + per - 1) // per
    words_max = PIPE_MAX_N * qbytes // 4
    kwords = (words_max + HALF - 1) // HALF
    stores = []
    for t in range(NARROW_THREADS):
        if NARROW_THREADS // wq >= 3:
            G = NARROW_THREADS // wq
            kw0 = t % wq if t < G * wq else wq
            rfirst = t // wq if t < G * wq else 0
            rstep = G
        else:
            kw0, rfirst, rstep = t % HALF, t // HALF, 2
        for j in range(kwords):
            k = kw0 + HALF * j
            if k >= wq:
                break
            assert per * k < n
            r = rfirst
            while r < rows:
                stores.append((r, k))
                r += rstep
            while r < R:
                stores.append((r, k))
                r += rstep
    return wq, stores


@pytest.mark.parametrize("qbytes", [1, 2])
def test_every_word_of_every_chunk_is_written_once(qbytes):
    checked = set()
    for stage in STAGES:
        for n in range(1, PIPE_MAX_N + 1):
            R = _chunk_rows(n, stage)
            if (n, R) in checked:
                continue
            checked.add((n, R))
            assert 1 <= R <= 32 and R * n * 4 <= stage and 32 % R == 0
            stride = (n * qbytes + 31) // 32 * 32          # pipe_row_stride
            for rows in sorted({1, R // 2 or 1, R - 1 or 1, R}):
                wq, stores = _writes(n, qbytes, rows, R)
                assert len(stores) == len(set(stores)), (n, R, rows)
                assert set(stores) == {(r, k) for r in range(R) for k in range(wq)}, (n, R, rows)
                assert all(4 * k + 4 <= stride for _, k in stores)


def test_short_rows_keep_most_threads_busy():
    """The reason for the row groups: at n = 100 (uint8, 25 words) 250 of the
    256 threads have a word, at n = 300 (75 words) 225; at n = 500 (125
    words, one thread per word position) 250."""
    for n, busy in ((100, 250), (300, 225), (500, 250)):
        wq = (n + 3) // 4
        if NARROW_THREADS // wq >= 3:
            got = (NARROW_THREADS // wq) * wq
        else:
            got = 2 * min(wq, HALF)
        assert got == busy, n


# --------------------------------------------------------------- predecessors
def test_pred_stage_model_follows_the_kernel_source():
    src = open(SRC).read()
    for line in ("static constexpr int W = 32 / (int)sizeof(PT);",
                 "const int sw = ((lane >> 2) & 3) << 1;",
                 "st[lane * 8 + ((pos >> 1) ^ sw)] = __byte_perm(pend, p, 0x5410);",
                 "st[lane * 8 + (pos ^ sw)] = p;",
                 "if (sizeof(PT) == 2 && (cnt & 1)) st[lane * 8 + ((cnt >> 1) ^ (((lane >> 2) & 3) << 1))] = pend;",
                 "if (wide && cnt == W) {",
                 "const int k2 = lane & 3;",
                 "const int r = 8 * m + (lane >> 2);",
                 "const int sz = ((r >> 2) & 3) << 1;",
                 "const uint2 v = *reinterpret_cast<const uint2*>(st + r * 8 + (2 * k2 ^ sz));",
                 "PT* dst = tile + (int64_t)r * n + (i0 - 1) + 2 * k2 * PER;",
                 "const int k = lane & 7;",
                 "const int r = 4 * m + (lane >> 3);",
                 "const uint32_t v = st[r * 8 + (k ^ ((m & 3) << 1))];",
                 "if (r < rows && k * PER < cnt) {",
                 "} else if (pairs && k * 2 + 1 < cnt) {",
                 "if (k * 2 + 1 < cnt) dst[1] = (PT)(v >> 16);",
                 "ps.pairs = sizeof(PT) == 4 || ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.pred) & 3) == 0);",
                 "ps.wide = (n % (8 / (int)sizeof(PT))) == 0 && (reinterpret_cast<uintptr_t>(a.pred) & 7) == 0;",
                 "if (u % W == W - 1) ps.flush(i - W + 1, W);",
                 "if (u % W == W - 1 || i == n) ps.flush(i - u % W, u % W + 1);"):
        assert line in src, line


def _pred_flush(size, cnt, rows, pairs, wide, n, i0, s0, base):
    """Stores of one flush: [(byte address, nbytes, [(row, position, value)])].
    Lane l's predecessor of position i0 + e is the code 1000 * l + e."""
    W, PER = 32 // size, 4 // size
    st = [[None] * 8 for _ in range(32)]
    for lane in range(32):
        sw = ((lane >> 2) & 3) << 1
        pend = None
        for pos in range(cnt):
            p = (lane, pos)
            if size == 2:
                if pos % 2 == 0:
                    pend = p
                else:
                    st[lane][(pos >> 1) ^ sw] = (pend, p)
            else:
                st[lane][pos ^ sw] = (p,)
        if size == 2 and cnt % 2:
            st[lane][(cnt >> 1) ^ sw] = (pend, None)
    stores = []

    def addr(r, col):
        return base + ((s0 + r) * n + (i0 - 1) + col) * size

    if wide and cnt == W:
        for lane in range(32):
            k2 = lane & 3
            for m in range(4):
                r = 8 * m + (lane >> 2)
                sz = ((r >> 2) & 3) << 1
                w = (2 * k2) ^ sz
                assert w % 2 == 0
                v = st[r][w] + st[r][w + 1]
                if r < rows:
                    stores.append((addr(r, 2 * k2 * PER), 8, [(r, 2 * k2 * PER + e, x)
                                                              for e, x in enumerate(v)]))
        return stores
    for lane in range(32):
        k = lane & 7
        for m in range(8):
            r = 4 * m + (lane >> 3)
            v = st[r][k ^ ((m & 3) << 1)]
            if r < rows and k * PER < cnt:
                col = k * PER
                if size == 4 or (pairs and k * 2 + 1 < cnt):
                    stores.append((addr(r, col), 4, [(r, col + e, x) for e, x in enumerate(v)]))
                else:
                    stores.append((addr(r, col), 2, [(r, col, v[0])]))
                    if k * 2 + 1 < cnt:
                        stores.append((addr(r, col + 1), 2, [(r, col + 1, v[1])]))
    return stores


@pytest.mark.parametrize("size", [2, 4])
def test_pred_stage_writes_each_position_once(size):
    """Every flush the kernel makes (a full block of W positions, or the last
    cnt at the end of the tour; W = 16 uint16 or 8 int32 predecessors)
    writes each (row, position) below (rows, cnt) once, with its own value,
    and each 4- or 8-byte store on its own alignment whenever the launch
    chose pairs / wide for that n and base address."""
    W = 32 // size
    for n in (W, 2 * W, 3 * W + 5, 100, 101, 500, 513):
        for base in (0, 2, 4, 8, 16):
            if base % size:
                continue
            pairs = size == 4 or (n % 2 == 0 and base % 4 == 0)
            wide = n % (8 // size) == 0 and base % 8 == 0
            for i0 in range(1, n + 1, W):
                cnt = min(W, n - i0 + 1)
                for rows in (1, 17, 32):
                    got = {}
                    for a, nb, elems in _pred_flush(size, cnt, rows, pairs, wide, n, i0, 64, base):
                        assert a % nb == 0, (n, base, i0, nb)
                        for r, pos, val in elems:
                            assert (r, pos) not in got
                            got[(r, pos)] = val
                    assert set(got) == {(r, p) for r in range(rows) for p in range(cnt)}
                    assert all(val == (r, p) for (r, p), val in got.items())

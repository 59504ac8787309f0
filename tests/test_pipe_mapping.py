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

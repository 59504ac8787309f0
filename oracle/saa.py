"""Oracle of the SAA candidate search over giant tours.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper scores
first-stage candidates by the sample-average-approximation mean of the
second-stage Split over the scenario set (Sec. "Decision Quality under Fixed
Time Budgets"; Tables tab:gpu_dsirp and tab:cand_cvrp count candidates
evaluated per time budget; its candidates come from a genetic algorithm).
The search written here proposes them by local search instead, with this
rule (the library's header states the same rule):

- iteration t starts from the current tour x and scores x and B neighbours;
- neighbour k takes z = SplitMix64 output number c = t*B + k of the stream
  `seed` (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014: the c-th output is the finaliser applied to
  seed + (c+1)*gamma, with the finaliser constants of Stafford's variant 13),
  a = (z mod 2^32) mod n, b = (z >> 40) mod (n-1), b += 1 if b >= a,
  kind = enabled[((z >> 32) & 255) mod len(enabled)] with the enabled kinds
  in the order 2-opt, relocate, swap;
- 2-opt reverses positions min(a,b)..max(a,b); relocate takes the customer at
  position a out and reinserts it to end at position b; swap exchanges the
  customers at a and b (0-based positions);
- every candidate's score is the FP64 Split mean over all scenarios
  (oracle.split); the lowest-scoring neighbour (the first one on ties)
  replaces x if its score is strictly below x's.

Candidate tours are built with list operations (slice reversal, pop/insert,
exchange), not with the library's per-position source map.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
KINDS = ("2opt", "relocate", "swap")


def splitmix64(seed: int, c: int) -> int:
    """Output number c (0-based) of the SplitMix64 stream seeded with seed."""
    z = (seed + (c + 1) * GAMMA) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def draw_move(seed: int, c: int, n: int, kinds=KINDS):
    """(kind, a, b) of move number c; 2-opt gives a < b."""
    enabled = [k for k in KINDS if k in kinds]
    z = splitmix64(seed, c)
    a = (z & 0xFFFFFFFF) % n
    b = (z >> 40) % (n - 1)
    if b >= a:
        b += 1
    kind = enabled[((z >> 32) & 0xFF) % len(enabled)]
    if kind == "2opt":
        a, b = min(a, b), max(a, b)
    return kind, a, b


def apply_move(tour, kind, a, b):
    """The neighbour of tour (a sequence of customers) under one move."""
    t = list(tour)
    if kind == "2opt":
        t[a:b + 1] = t[a:b + 1][::-1]
    elif kind == "relocate":
        x = t.pop(a)
        t.insert(b, x)
    elif kind == "swap":
        t[a], t[b] = t[b], t[a]
    else:
        raise ValueError(kind)
    return t


def saa_search(tour0, Q, demands, coords, B, iters, seed, kinds=KINDS, t0=0,
               split=None):
    """Runs iterations t0 .. t0+iters-1 from tour0.  Returns a dict:
    tour (final), trace [iters] (best score after each iteration), accepted
    [iters] (neighbour index or -1), means [iters][B+1] (score of the start
    tour of the iteration, then of each neighbour), cands [iters] (the
    neighbours, int32 [B, n] each)."""
    if split is None:
        from oracle import split as _split
        split = _split
    n = len(tour0)
    x = [int(v) for v in tour0]
    trace, accepted, means, allc = [], [], [], []

    def score(t):
        return split(np.asarray(t, np.int32), Q, demands, coords=coords,
                     want_pred=False)["mean"]

    for t in range(t0, t0 + iters):
        cands = [apply_move(x, *draw_move(seed, t * B + k, n, kinds)) for k in range(B)]
        m0 = score(x)
        ms = [score(c) for c in cands]
        kbest = int(np.argmin(ms))  # first minimum
        take = ms[kbest] < m0
        if take:
            x = cands[kbest]
        trace.append(ms[kbest] if take else m0)
        accepted.append(kbest if take else -1)
        means.append([m0] + ms)
        allc.append(np.asarray(cands, np.int32))
    return {"tour": np.asarray(x, np.int32), "trace": np.asarray(trace),
            "accepted": np.asarray(accepted, np.int32), "means": np.asarray(means),
            "cands": allc}

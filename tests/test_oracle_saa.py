"""Pins of the SAA candidate-search oracle: the move generator against
SplitMix64's published known-answer outputs, the moves against their
inverses, and the search's choices against a brute-force scan of the whole
neighbourhood."""
import itertools

import numpy as np
import pytest

import oracle
from tests.golden_io import load

KINDS = ("2opt", "relocate", "swap")


def test_splitmix64_known_answer():
    g = load("splitmix64_1234567.json")
    assert [oracle.splitmix64(g["seed"], c) for c in range(5)] == g["outputs"]


@pytest.mark.parametrize("n", [2, 3, 7, 100])
def test_draws_are_valid_moves(n):
    counts = dict.fromkeys(KINDS, 0)
    for c in range(3000):
        kind, a, b = oracle.draw_move(99, c, n)
        assert 0 <= a < n and 0 <= b < n and a != b
        if kind == "2opt":
            assert a < b
        counts[kind] += 1
    for k in KINDS:  # each kind about a third of the draws
        assert 800 < counts[k] < 1200
    for kinds in (("swap",), ("2opt", "swap"), ("relocate",)):
        assert {oracle.draw_move(5, c, n, kinds)[0] for c in range(200)} <= set(kinds)


def test_moves_are_permutations_with_inverses():
    rng = np.random.default_rng(0)
    for trial in range(300):
        n = int(rng.integers(2, 30))
        t = list(rng.permutation(n) + 1)
        kind, a, b = oracle.draw_move(int(rng.integers(1 << 62)), trial, n)
        u = oracle.apply_move(t, kind, a, b)
        assert sorted(u) == sorted(t) and u != t
        back = {"2opt": (a, b), "relocate": (b, a), "swap": (a, b)}[kind]
        assert oracle.apply_move(u, kind, *back) == t


def test_moves_by_hand():
    t = [1, 2, 3, 4, 5, 6]
    assert oracle.apply_move(t, "2opt", 1, 4) == [1, 5, 4, 3, 2, 6]
    assert oracle.apply_move(t, "relocate", 1, 4) == [1, 3, 4, 5, 2, 6]
    assert oracle.apply_move(t, "relocate", 4, 1) == [1, 5, 2, 3, 4, 6]
    assert oracle.apply_move(t, "swap", 0, 5) == [6, 2, 3, 4, 5, 1]


def _instance(seed, n, S, Q, lam):
    rng = np.random.default_rng(seed)
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50, 50)
    xy[1:] = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    q = np.clip(rng.poisson(lam, (S, n)), 1, Q).astype(np.int32)
    tour0 = (rng.permutation(n) + 1).astype(np.int32)
    return tour0, xy, q


def _score(t, Q, q, xy):
    return oracle.split(np.asarray(t, np.int32), Q, q, coords=xy, want_pred=False)["mean"]


def test_search_bookkeeping():
    tour0, xy, q = _instance(1, 9, 30, 20, 5.0)
    r = oracle.saa_search(tour0, 20, q, xy, B=12, iters=8, seed=7)
    tr, acc, ms = r["trace"], r["accepted"], r["means"]
    assert np.all(np.diff(tr) <= 0)
    for t in range(8):
        if acc[t] >= 0:
            assert ms[t][1 + acc[t]] == tr[t] < ms[t][0]
            assert ms[t][1 + acc[t]] == ms[t][1:].min()
        else:
            assert ms[t][1:].min() >= ms[t][0] == tr[t]
        if t + 1 < 8:
            assert ms[t + 1][0] == tr[t]
    assert _score(r["tour"], 20, q, xy) == tr[-1]
    # continuing from iteration 5 reproduces the tail of the trajectory
    r5 = oracle.saa_search(tour0, 20, q, xy, B=12, iters=5, seed=7)
    r3 = oracle.saa_search(r5["tour"], 20, q, xy, B=12, iters=3, seed=7, t0=5)
    np.testing.assert_array_equal(r3["trace"], tr[5:])
    np.testing.assert_array_equal(r3["tour"], r["tour"])


def test_search_ends_in_a_local_optimum():
    """n = 4: 24 tours and 24 moves (6 2-opt, 12 relocate, 6 swap).  With 400
    draws per iteration every move is drawn, so the search is steepest
    descent: its last tour has no strictly better neighbour, and its first
    step takes the best neighbour of the start tour (both checked by
    enumerating the neighbourhood)."""
    tour0, xy, q = _instance(2, 4, 40, 12, 4.0)
    Q = 12
    r = oracle.saa_search(tour0, Q, q, xy, B=400, iters=6, seed=3)

    def neighbourhood(t):
        out = []
        for a, b in itertools.permutations(range(4), 2):
            if a < b:
                out.append(oracle.apply_move(t, "2opt", a, b))
                out.append(oracle.apply_move(t, "swap", a, b))
            out.append(oracle.apply_move(t, "relocate", a, b))
        return out

    best0 = min(_score(u, Q, q, xy) for u in neighbourhood(list(tour0)))
    s0 = _score(tour0, Q, q, xy)
    assert r["trace"][0] == min(best0, s0)
    final = _score(r["tour"], Q, q, xy)
    assert all(_score(u, Q, q, xy) >= final for u in neighbourhood(list(r["tour"])))
    allbest = min(_score(p, Q, q, xy) for p in itertools.permutations(range(1, 5)))
    assert final >= allbest


def test_draws_worked_from_the_published_outputs():
    """The draw rule worked by hand on the SplitMix64 known-answer outputs of
    state 1234567 (tests/golden/splitmix64_1234567.json).  Output 0, z =
    6457827717110365317: low word 4211670149, z >> 40 = 5873360, byte
    (z >> 32) & 255 = 23.  Output 1, z = 3203168211198807973: 1481904037,
    2913264, 132.  Output 2, z = 9817491932198370423: 2750577783, 8928956,
    229.  a = low word mod n; b = (z >> 40) mod (n - 1), plus one when b >= a;
    kind = byte mod (kinds enabled), in the order 2-opt, relocate, swap;
    2-opt orders a < b."""
    s = load("splitmix64_1234567.json")["seed"]
    assert oracle.draw_move(s, 0, 10) == ("swap", 9, 5)       # 23 mod 3 = 2; b = 5 < a
    assert oracle.draw_move(s, 0, 7) == ("swap", 1, 3)        # a = 1; b = 2 >= a -> 3
    assert oracle.draw_move(s, 1, 10) == ("2opt", 0, 7)       # 132 mod 3 = 0; (7, 0) ordered
    assert oracle.draw_move(s, 1, 7) == ("2opt", 0, 5)        # a = 5, b = 0
    assert oracle.draw_move(s, 2, 10) == ("relocate", 3, 2)   # 229 mod 3 = 1; b = 2 < a = 3
    assert oracle.draw_move(s, 2, 7) == ("relocate", 2, 3)    # a = 2; b = 2 >= a -> 3
    two = ("2opt", "swap")
    assert oracle.draw_move(s, 0, 10, two) == ("swap", 9, 5)  # 23 mod 2 = 1
    assert oracle.draw_move(s, 1, 10, two) == ("2opt", 0, 7)  # 132 mod 2 = 0
    assert oracle.draw_move(s, 2, 10, two) == ("swap", 3, 2)  # 229 mod 2 = 1


def _ray_instance(seed, n, S):
    """Customers on a ray from the depot at integer distances (3, 6, ...):
    every travel cost is an exact integer, so every score is exact and equal
    scores are exact ties.  Q holds every scenario's whole demand."""
    rng = np.random.default_rng(seed)
    xy = np.zeros((n + 1, 2), np.float32)
    xy[1:, 0] = 3.0 * (rng.permutation(n) + 1)
    q = rng.integers(1, 4, size=(S, n)).astype(np.int32)
    return xy, q, int(q.sum(axis=1).max()), (np.argsort(xy[1:, 0]) + 1).astype(np.int32)


def test_search_accepts_strict_improvements_only():
    """The tour out along the ray scores 2 max x, the least any tour can; many
    of its neighbours (a suffix reversed, a customer moved to the way back)
    score exactly that too.  A neighbour replaces the current tour only when
    strictly better, so none is taken."""
    xy, q, Q, out = _ray_instance(5, 6, 4)
    r = oracle.saa_search(out, Q, q, xy, 30, 3, 11)
    m = r["means"]
    assert (r["accepted"] == -1).all() and list(r["tour"]) == list(out)
    assert (m[:, 1:] >= m[:, :1]).all()
    assert (m[:, 1:] == m[:, :1]).sum() >= 3          # exact ties with the current tour
    assert np.array_equal(r["trace"], m[:, 0])


def test_search_takes_the_first_of_equal_best_neighbours():
    """From a zigzag tour along the ray several neighbours often reach the
    same best score (one move drawn twice, or two moves giving tours of equal
    cost); the accepted neighbour must be the first of them."""
    xy, q, Q, out = _ray_instance(6, 6, 4)
    zig = out[[0, 5, 1, 4, 2, 3]]
    r = oracle.saa_search(zig, Q, q, xy, 40, 4, 12)
    tied_and_taken = 0
    for t in range(4):
        m0, ms = r["means"][t][0], list(r["means"][t][1:])
        best = min(ms)
        first = ms.index(best)
        assert r["accepted"][t] == (first if best < m0 else -1), t
        tied_and_taken += best < m0 and ms.count(best) > 1
    assert tied_and_taken >= 1

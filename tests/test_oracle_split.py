"""Pins of the Split oracle (Eq. eqdpA) against what the paper and the
mathematics fix: the paper's worked example, the figure example's capacity
masks, brute-force enumeration of every split, closed forms and invariants,
and central finite differences for the arc-usage gradient."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests import brute
from tests.golden_io import arr, load


def _dist_from(c):
    return np.asarray(c, dtype=np.float32)


# ---------------------------------------------------------------- worked example
def test_split_toy_matrix_and_values():
    g = load("split_toy.json")
    dist = _dist_from(g["cost_matrix"])
    tour = arr(g["tour"], np.int32)
    q = arr(g["demand_by_customer"], np.int32)
    A, V = oracle.split_matrix(tour, g["Q"], q, dist=dist)
    np.testing.assert_array_equal(A, arr(g["A"]))
    np.testing.assert_array_equal(V, arr(g["V"]))
    r = oracle.split(tour, g["Q"], q[None, :], dist=dist, want_margin=True)
    assert r["cost"][0] == g["V"][-1]
    np.testing.assert_array_equal(r["pred"][0], arr(g["pred"], np.int32))
    # feasible arcs: (0,1), (0,2), (1,2), (2,3)
    assert r["arcs"][0] == 4


def test_split_figure_feasibility():
    g = load("split_figure_feasibility.json")
    tour = arr(g["tour"], np.int32)
    n = len(tour)
    # customers all at one point away from the depot: route cost = 2 per route,
    # so the optimum is the minimum number of capacity-feasible routes.
    dist = np.zeros((n + 1, n + 1), np.float32)
    dist[0, 1:] = 1.0
    dist[1:, 0] = 1.0
    for sc in g["scenarios"]:
        q = arr(sc["demand_by_customer"], np.int32)
        A, V = oracle.split_matrix(tour, g["Q"], q, dist=dist)
        pos = {c: k + 1 for k, c in enumerate(g["tour"])}
        for route in sc["routes"]:
            p = pos[route[0]] - 1
            i = pos[route[-1]]
            assert [g["tour"][k] for k in range(p, i)] == route
            assert np.isfinite(A[p, i]), route       # capacity-feasible
        r = oracle.split(tour, g["Q"], q[None, :], dist=dist)
        assert r["cost"][0] == 2.0 * sc["min_routes"]


# ---------------------------------------------------------------- brute force
def _rand_instance(rng, n, Q, qmax, dist_mode):
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50.0, 50.0)
    xy[1:] = rng.uniform(0, 100, size=(n, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, qmax + 1, size=n).astype(np.int32)
    if dist_mode:
        d = rng.uniform(1, 100, size=(n + 1, n + 1)).astype(np.float32)  # asymmetric, non-metric
        np.fill_diagonal(d, 0)
        return tour, None, d, q
    return tour, xy, None, q


@pytest.mark.parametrize("seed", range(40))
def test_split_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(0, 11))
    Q = int(rng.integers(1, 40))
    dist_mode = bool(seed % 2)
    tour, xy, d, q = _rand_instance(rng, n, Q, qmax=Q + 3 if seed % 5 == 0 else Q // 2 + 1,
                                    dist_mode=dist_mode)
    if dist_mode:
        cost = lambda a, b: float(d[a, b])
    else:
        cost = lambda a, b: brute.euclid(xy, a, b)
    best, parts = brute.split_brute(list(tour), list(q), Q, cost)
    r = oracle.split(tour, Q, q[None, :], coords=xy, dist=d, want_margin=True)
    c = r["cost"][0]
    if math.isinf(best):
        assert math.isinf(c)
        return
    assert abs(c - best) <= 1e-12 * max(1.0, abs(best))
    # explicit-matrix DP agrees with the windowed recursion
    _, V = oracle.split_matrix(tour, Q, q, coords=xy, dist=d)
    assert abs(V[-1] - c) <= 1e-12 * max(1.0, abs(c))
    # the backtracked routes are one of the optimal partitions when unique
    if n and len(parts) == 1:
        pred = r["pred"][0]
        routes, i = [], n
        while i > 0:
            p = int(pred[i - 1])
            routes.append([int(x) for x in tour[p:i]])
            i = p
        assert routes[::-1] == parts[0]
    # arcs = number of capacity-feasible pairs p < i
    L = np.concatenate([[0], np.cumsum(q[tour - 1])]) if n else np.zeros(1)
    narcs = sum(1 for i in range(1, n + 1) for p in range(i) if L[i] - L[p] <= Q)
    assert r["arcs"][0] == narcs


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", range(5))
def test_split_every_demand_equals_Q(seed):
    rng = np.random.default_rng(seed)
    n, Q = 30, 17
    tour, xy, _, _ = _rand_instance(rng, n, Q, Q, False)
    q = np.full(n, Q, np.int32)
    r = oracle.split(tour, Q, q[None, :], coords=xy)
    expect = sum(brute.euclid(xy, 0, c) + brute.euclid(xy, c, 0) for c in tour)
    assert abs(r["cost"][0] - expect) <= 1e-12 * expect
    np.testing.assert_array_equal(r["pred"][0], np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("seed", range(5))
def test_split_single_route_is_closed_tour(seed):
    """Euclidean costs, total demand <= Q: by the triangle inequality no split
    beats the single route, whose cost is the closed tour through the depot."""
    rng = np.random.default_rng(10 + seed)
    n = 40
    tour, xy, _, _ = _rand_instance(rng, n, 1, 1, False)
    q = rng.integers(1, 5, size=n).astype(np.int32)
    Q = int(q.sum())
    r = oracle.split(tour, Q, q[None, :], coords=xy)
    expect = brute.euclid(xy, 0, tour[0]) + brute.euclid(xy, tour[-1], 0)
    expect += sum(brute.euclid(xy, a, b) for a, b in zip(tour[:-1], tour[1:]))
    assert abs(r["cost"][0] - expect) <= 1e-12 * expect
    assert r["pred"][0][-1] == 0


def test_split_degenerate_sizes():
    xy = np.array([[50, 50], [53, 54]], np.float32)
    r = oracle.split(np.array([1], np.int32), 10, np.array([[4]], np.int32), coords=xy)
    assert r["cost"][0] == pytest.approx(10.0, abs=1e-12)
    r0 = oracle.split(np.zeros(0, np.int32), 10, np.zeros((3, 0), np.int32),
                      coords=np.array([[50, 50]], np.float32))
    np.testing.assert_array_equal(r0["cost"], np.zeros(3))
    # a demand above Q makes the scenario infeasible: +inf, preds -1 from there
    r1 = oracle.split(np.array([1], np.int32), 10, np.array([[11]], np.int32), coords=xy)
    assert math.isinf(r1["cost"][0]) and r1["pred"][0][0] == -1
    assert math.isinf(r1["mean"])


# ---------------------------------------------------------------- invariants
def test_split_monotone_in_Q_and_prefix():
    rng = np.random.default_rng(7)
    n = 60
    tour, xy, _, _ = _rand_instance(rng, n, 1, 1, False)
    q = rng.integers(1, 20, size=(8, n)).astype(np.int32)
    prev = None
    for Q in (19, 25, 40, 80, 200, 2000):
        c = oracle.split(tour, Q, q, coords=xy)["cost"]
        if prev is not None:
            assert np.all(c <= prev + 1e-9)
        prev = c
    # metric costs: J(i) is non-decreasing in i
    _, V = oracle.split_matrix(tour, 40, q[0], coords=xy)
    assert np.all(np.diff(V) >= -1e-9)


def test_split_margin_definition():
    rng = np.random.default_rng(3)
    n = 25
    tour, xy, _, q = _rand_instance(rng, n, 30, 10, False)
    r = oracle.split(tour, 30, q[None, :], coords=xy, want_margin=True)
    A, V = oracle.split_matrix(tour, 30, q, coords=xy)
    for i in range(1, n + 1):
        cands = sorted(V[p] + A[p, i] for p in range(i) if np.isfinite(A[p, i]))
        if len(cands) < 2:
            assert math.isinf(r["margin"][0][i - 1])
        else:
            assert r["margin"][0][i - 1] == pytest.approx((cands[1] - cands[0]) / abs(cands[0]),
                                                          rel=1e-9, abs=1e-15)


def test_split_ties_and_infeasible_positions_by_brute_force():
    """Readings S3 and S4: with travel costs of 0, 1 or 2 every route cost
    and every sum of them is exact, so ties between predecessors are exact.
    pred(i) must be the smallest p among the optimal candidates for J(i)
    that brute force lists (each candidate = the best split of the first p
    customers plus the route s_{p+1..i}), and -1 at every position that no
    feasible split reaches (a demand above Q at or before it)."""
    ties = unreachable = 0
    for seed in range(30):
        rng = np.random.default_rng(2700 + seed)
        n = int(rng.integers(2, 9))
        Q = int(rng.integers(2, 8))
        d = rng.integers(0, 3, size=(n + 1, n + 1)).astype(np.float32)
        np.fill_diagonal(d, 0.0)
        tour = (rng.permutation(n) + 1).astype(np.int32)
        q = rng.integers(0, Q + 1, size=n).astype(np.int32)
        if seed % 3 == 0:
            q[tour[int(rng.integers(0, n))] - 1] = Q + 1
        r = oracle.split(tour, Q, q[None, :], dist=d)
        pred = r["pred"][0]
        for i in range(1, n + 1):
            cands = brute.split_candidates(list(tour), list(q), Q,
                                           lambda a, b: float(d[a, b]), i)
            if not cands:
                unreachable += 1
                assert pred[i - 1] == -1, (seed, i)
                continue
            best = min(v for v, _ in cands)
            opt = [p for v, p in cands if v == best]
            ties += len(opt) > 1
            assert pred[i - 1] == min(opt), (seed, i, opt)
        assert math.isinf(r["cost"][0]) == (seed % 3 == 0)
    assert ties >= 10 and unreachable >= 10


def test_route_counts_skip_infeasible_scenarios():
    """A scenario with no feasible split (a demand above Q: predecessors -1
    from there on) contributes no route and is counted as skipped; the counts
    are those of the feasible scenarios alone, and their total is the number
    of routes found by walking each feasible scenario's predecessors back."""
    rng = np.random.default_rng(41)
    n, Q, S = 25, 30, 40
    tour, xy, _, _ = _rand_instance(rng, n, Q, 10, False)
    q = rng.integers(1, 11, size=(S, n)).astype(np.int32)
    bad = [3, 17, 18, 39]
    for s in bad:
        q[s, int(rng.integers(0, n))] = Q + 1
    r = oracle.split(tour, Q, q, coords=xy)
    start, end, skipped = oracle.split_route_counts(r["pred"])
    assert skipped == len(bad)
    keep = np.setdiff1d(np.arange(S), bad)
    s2, e2, k2 = oracle.split_route_counts(r["pred"][keep])
    assert k2 == 0 and np.array_equal(start, s2) and np.array_equal(end, e2)
    routes = 0
    for s in keep:
        i = n
        while i > 0:
            i = int(r["pred"][s][i - 1])
            routes += 1
    assert start.sum() == end.sum() == routes


# ---------------------------------------------------------------- gradient
def test_split_gradient_identities_and_fd():
    """d mean / d dist from backtracked arc usage equals central finite
    differences of the FP64 mean (piecewise linear: exact at tie-free points)."""
    spec = wl.SplitSpec("t", 40, 60, 64, 11, "poisson", lam=10.0, lo=1, hi=60, dist_mode=True)
    tour, xy, dist = wl.split_tour(spec)
    q = wl.split_demands(spec)
    r = oracle.split(tour, spec.Q, q, dist=dist)
    g = oracle.split_mean_grad(tour, r["pred"])
    n = spec.n
    # identities per scenario (each customer continues its route or ends it)
    assert g[0, tour[0]] == pytest.approx(1.0)
    assert g[tour[-1], 0] == pytest.approx(1.0)
    for k in range(n - 1):
        assert g[tour[k], tour[k + 1]] + g[tour[k], 0] == pytest.approx(1.0)
    start, end, skipped = oracle.split_route_counts(r["pred"])
    assert skipped == 0 and start.sum() == end.sum()
    for k in range(n):
        assert g[0, tour[k]] * spec.S == pytest.approx(start[k])
        assert g[tour[k], 0] * spec.S == pytest.approx(end[k])
    # central finite differences on structurally nonzero + random zero entries
    h = 1e-3
    rng = np.random.default_rng(0)
    entries = [(0, int(c)) for c in tour] + [(int(c), 0) for c in tour]
    entries += [(int(a), int(b)) for a, b in zip(tour[:-1], tour[1:])]
    entries += [tuple(int(v) for v in rng.integers(1, n + 1, 2)) for _ in range(30)]
    checked = 0
    for (a, b) in entries:
        dp = dist.copy(); dp[a, b] += h
        dm = dist.copy(); dm[a, b] -= h
        rp = oracle.split(tour, spec.Q, q, dist=dp)
        rm = oracle.split(tour, spec.Q, q, dist=dm)
        if not (np.array_equal(rp["pred"], r["pred"]) and np.array_equal(rm["pred"], r["pred"])):
            continue  # a tie within h: gradient not defined there
        # the fp32 perturbation actually applied
        hp = float(np.float32(dist[a, b] + np.float32(h))) - float(dist[a, b])
        hm = float(dist[a, b]) - float(np.float32(dist[a, b] - np.float32(h)))
        fd = (rp["mean"] - rm["mean"]) / (hp + hm)
        assert fd == pytest.approx(g[a, b], abs=1e-9), (a, b)
        checked += 1
    assert checked >= len(entries) // 2


# ---------------------------------------------------------------- workloads
def test_split_workload_c1_smoke():
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    q = wl.split_demands(spec)
    assert q.shape == (spec.S, spec.n) and q.min() >= 1 and q.max() <= spec.Q
    r = oracle.split(tour, spec.Q, q, coords=xy)
    assert np.all(np.isfinite(r["cost"]))
    assert abs(r["mean"] - r["cost"].mean()) <= 1e-9 * r["mean"]
    # a seeded estimate over 200 scenarios gives about 439 feasible arcs each
    assert 300 < r["arcs"].mean() < 600

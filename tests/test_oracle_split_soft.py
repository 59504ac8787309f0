"""Pins of the soft-capacity Split oracle (every split allowed, beta per unit
of route load above Q -- the penalised load of the paper's CVRPSD model)
against brute-force enumeration of every split, closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle
from tests import brute


def _instance(rng, n, qmax, dist_mode):
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
def test_soft_split_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(1, 11))
    Q = int(rng.integers(1, 40))
    beta = float(rng.choice([0.0, 0.3, 2.0, 15.0, 1e3]))
    dist_mode = bool(seed % 2)
    tour, xy, d, q = _instance(rng, n, qmax=Q + 8, dist_mode=dist_mode)
    cost = (lambda a, b: float(d[a, b])) if dist_mode else (lambda a, b: brute.euclid(xy, a, b))
    best, parts = brute.split_soft_brute(list(tour), list(q), Q, beta, cost)
    r = oracle.split_soft(tour, Q, beta, q[None, :], coords=xy, dist=d)
    c = r["cost"][0]
    assert math.isfinite(c)
    assert abs(c - best) <= 1e-12 * max(1.0, abs(best))
    if len(parts) == 1:  # the backtracked routes are the unique optimum
        pred = r["pred"][0]
        routes, i = [], n
        while i > 0:
            p = int(pred[i - 1])
            routes.append([int(x) for x in tour[p:i]])
            i = p
        assert routes[::-1] == parts[0]
    assert r["arcs"][0] == n * (n + 1) // 2  # every pair (p, i)


@pytest.mark.parametrize("seed", range(5))
def test_soft_split_without_penalty_is_closed_tour(seed):
    """beta = 0: capacity costs nothing, and with Euclidean costs (triangle
    inequality) no cut beats the single route: the closed tour."""
    rng = np.random.default_rng(20 + seed)
    n = 40
    tour, xy, _, q = _instance(rng, n, 30, False)
    r = oracle.split_soft(tour, 10, 0.0, q[None, :], coords=xy)
    expect = brute.euclid(xy, 0, tour[0]) + brute.euclid(xy, tour[-1], 0)
    expect += sum(brute.euclid(xy, a, b) for a, b in zip(tour[:-1], tour[1:]))
    assert abs(r["cost"][0] - expect) <= 1e-12 * expect
    assert r["pred"][0][-1] == 0


@pytest.mark.parametrize("seed", range(4))
def test_soft_split_equals_hard_when_no_route_can_overflow(seed):
    """Q >= the total demand: no route ever exceeds Q, so the penalty is never
    charged and the soft DP is the hard DP, operation for operation."""
    rng = np.random.default_rng(30 + seed)
    n, S = 25, 20
    tour, xy, _, _ = _instance(rng, n, 1, False)
    q = rng.integers(0, 9, size=(S, n)).astype(np.int32)
    Q = int(q.sum(axis=1).max())
    h = oracle.split(tour, Q, q, coords=xy)
    s = oracle.split_soft(tour, Q, 7.5, q, coords=xy)
    np.testing.assert_array_equal(s["cost"], h["cost"])
    np.testing.assert_array_equal(s["pred"], h["pred"])


def test_soft_split_invariants():
    """Allowing overloaded routes never costs more than forbidding them; the
    cost is non-decreasing in beta, non-increasing in Q, and finite even
    when a single demand exceeds Q (where the hard DP is infeasible)."""
    rng = np.random.default_rng(41)
    n, S = 30, 60
    tour, xy, _, _ = _instance(rng, n, 1, False)
    q = rng.integers(1, 20, size=(S, n)).astype(np.int32)
    q[0, 3] = 90
    Q = 40
    hard = oracle.split(tour, Q, q, coords=xy)["cost"]
    prev = None
    for beta in (0.0, 0.5, 2.0, 10.0, 100.0, 1e4):
        soft = oracle.split_soft(tour, Q, beta, q, coords=xy)["cost"]
        assert np.all(np.isfinite(soft))
        fin = np.isfinite(hard)
        assert np.all(soft[fin] <= hard[fin] * (1 + 1e-12))
        if prev is not None:
            assert np.all(soft >= prev - 1e-9 * np.abs(prev))
        prev = soft
    assert math.isinf(hard[0])
    prevQ = None
    for Qv in (10, 20, 40, 80):
        c = oracle.split_soft(tour, Qv, 3.0, q, coords=xy)["cost"]
        if prevQ is not None:
            assert np.all(c <= prevQ + 1e-9 * np.abs(prevQ))
        prevQ = c


def test_soft_split_large_penalty_reaches_hard_optimum():
    """Integer demands: any overloaded route carries at least one unit of
    excess, and cutting it at every customer costs at most n * 2 * (largest
    depot distance) more; a larger beta makes every overload lose, so the
    soft optimum is the hard one whenever the hard problem is feasible."""
    rng = np.random.default_rng(52)
    n, S = 20, 30
    tour, xy, _, _ = _instance(rng, n, 1, False)
    q = rng.integers(1, 12, size=(S, n)).astype(np.int32)
    Q = 20
    dmax = max(brute.euclid(xy, 0, c) for c in range(1, n + 1))
    beta = 2.0 * n * 2.0 * dmax + 1.0
    h = oracle.split(tour, Q, q, coords=xy)
    s = oracle.split_soft(tour, Q, beta, q, coords=xy)
    np.testing.assert_allclose(s["cost"], h["cost"], rtol=1e-12)


@pytest.mark.parametrize("seed", range(12))
def test_soft_split_margin_by_brute_force(seed):
    """The margin of each position (relative gap between the best and the
    second-best predecessor, which decides where the GPU's predecessors are
    compared bit for bit) equals the gap between the two smallest candidate
    values of J(i), each built by brute force over the prefix splits."""
    rng = np.random.default_rng(5600 + seed)
    n = int(rng.integers(2, 9))
    Q = int(rng.integers(3, 30))
    beta = float(rng.choice([0.0, 0.7, 4.0, 50.0]))
    dist_mode = bool(seed % 2)
    tour, xy, d, q = _instance(rng, n, qmax=Q + 5, dist_mode=dist_mode)
    cost = (lambda a, b: float(d[a, b])) if dist_mode else (lambda a, b: brute.euclid(xy, a, b))
    r = oracle.split_soft(tour, Q, beta, q[None, :], coords=xy, dist=d, want_margin=True)
    for i in range(1, n + 1):
        vals = sorted(v for v, _ in brute.split_candidates(list(tour), list(q), Q, cost, i, beta))
        m = r["margin"][0][i - 1]
        if len(vals) < 2:
            assert math.isinf(m)
        else:
            assert m == pytest.approx((vals[1] - vals[0]) / abs(vals[0]), rel=1e-9, abs=1e-12), i


def test_soft_split_ties_by_brute_force():
    """Reading S4 for soft capacity: with travel costs of 0, 1 or 2 and an
    integer penalty every candidate value is exact, so ties are exact; pred(i)
    must be the smallest p among the optimal candidates for J(i) that brute
    force lists (every route allowed, beta per unit of load above Q)."""
    ties = overloaded = 0
    for seed in range(30):
        rng = np.random.default_rng(2750 + seed)
        n = int(rng.integers(2, 9))
        Q = int(rng.integers(1, 7))
        beta = float(rng.integers(1, 4))
        d = rng.integers(0, 3, size=(n + 1, n + 1)).astype(np.float32)
        np.fill_diagonal(d, 0.0)
        tour = (rng.permutation(n) + 1).astype(np.int32)
        q = rng.integers(0, Q + 3, size=n).astype(np.int32)
        overloaded += int((q > Q).any())
        r = oracle.split_soft(tour, Q, beta, q[None, :], dist=d)
        pred = r["pred"][0]
        for i in range(1, n + 1):
            cands = brute.split_candidates(list(tour), list(q), Q,
                                           lambda a, b: float(d[a, b]), i, beta=beta)
            best = min(v for v, _ in cands)
            opt = [p for v, p in cands if v == best]
            ties += len(opt) > 1
            assert pred[i - 1] == min(opt), (seed, i, opt)
    assert ties >= 20 and overloaded >= 10


def test_soft_split_mean_is_the_sample_average():
    """The mean is the average of the per-scenario costs over all S (the SAA
    mean); with soft capacity every scenario is finite."""
    rng = np.random.default_rng(2950)
    tour, xy, _, _ = _instance(rng, 20, 10, False)
    q = rng.integers(0, 25, size=(64, 20)).astype(np.int32)
    r = oracle.split_soft(tour, 30, 7.0, q, coords=xy)
    assert np.isfinite(r["cost"]).all()
    assert r["mean"] == pytest.approx(math.fsum(r["cost"]) / len(r["cost"]), rel=1e-14)

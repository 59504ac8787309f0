"""Pins of the fleet-limited Split oracle (at most K routes: Appendix A,
constraint eq:fleet_size; hard capacity as in Eq. eqdpA).

What fixes it, independently of the oracle's own code:
  - brute force over every set of cut points of the giant tour with at most K
    routes (tests/brute.py), n <= 9, random capacities, some infeasible;
  - the paper's giant-tour example (tour (1,2,4,3,5), Q = 17): the minimum
    numbers of routes it prints make K below them infeasible and K at them
    feasible;
  - closed forms: K = 1 is the closed tour when the total demand fits, else
    infeasible; K >= n is the unlimited Split; every demand = Q needs n routes;
  - the cost is non-increasing in K.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.brute import euclid, split_brute
from tests.golden_io import load


def _inst(seed, n, S, Q, qhi):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0, 100, (n + 1, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, qhi + 1, size=(S, n)).astype(np.int32)
    return tour, xy, q


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_fleet_matches_brute_force(seed, K):
    n = 3 + seed
    tour, xy, q = _inst(100 + seed, n, 12, 20, 14)
    q[0, 0] = 21  # one customer above Q: infeasible for every K
    o = oracle.split_fleet(tour, 20, K, q, coords=xy, want_margin=True)
    cost = lambda a, b: euclid(xy, a, b)
    for s in range(q.shape[0]):
        best, args = split_brute(tour.tolist(), q[s].tolist(), 20, cost, max_routes=K)
        if math.isinf(best):
            assert math.isinf(o["cost"][s]) and o["nroutes"][s] == 0
            assert (o["route"][s] == -1).all()
            continue
        assert abs(o["cost"][s] - best) <= 1e-12 * max(1.0, best)
        if len(args) == 1 and o["margin"][s] > 1e-9:
            routes = args[0]
            assert o["nroutes"][s] == len(routes)
            want = np.concatenate([[r] * len(rt) for r, rt in enumerate(routes)])
            assert np.array_equal(o["route"][s], want)


def test_fleet_paper_example_minimum_routes():
    """The example's scenarios need 3 and 2 routes: with fewer vehicles the
    oracle finds no split, with that many it finds one, and the split it
    returns uses at least that many routes."""
    g = load("split_figure_feasibility.json")
    tour = np.asarray(g["tour"], np.int32)
    rng = np.random.default_rng(3)
    xy = rng.uniform(0, 100, (len(tour) + 1, 2)).astype(np.float32)
    for sc in g["scenarios"]:
        q = np.asarray(sc["demand_by_customer"], np.int32)[None, :]
        m = sc["min_routes"]
        lo = oracle.split_fleet(tour, g["Q"], m - 1, q, coords=xy) if m > 1 else None
        if lo is not None:
            assert math.isinf(lo["cost"][0]) and lo["nroutes"][0] == 0
        ok = oracle.split_fleet(tour, g["Q"], m, q, coords=xy)
        assert math.isfinite(ok["cost"][0]) and ok["nroutes"][0] == m
        three = oracle.split_fleet(tour, g["Q"], 3, q, coords=xy)  # "three vehicles available"
        assert math.isfinite(three["cost"][0]) and m <= three["nroutes"][0] <= 3


def test_fleet_closed_forms():
    n, S, Q = 12, 40, 50
    tour, xy, q = _inst(7, n, S, Q, 8)
    # K = 1: the closed tour when everything fits, else no split
    one = oracle.split_fleet(tour, Q, 1, q, coords=xy)
    tsp = euclid(xy, 0, tour[0]) + euclid(xy, tour[-1], 0) + sum(
        euclid(xy, a, b) for a, b in zip(tour[:-1], tour[1:]))
    fits = q.sum(1) <= Q
    assert fits.any() and (~fits).any()
    np.testing.assert_allclose(one["cost"][fits], tsp, rtol=1e-12)
    assert np.isinf(one["cost"][~fits]).all()
    assert (one["nroutes"][fits] == 1).all()
    # K >= n: the unlimited Split, bit for bit (the same FP64 sums)
    full = oracle.split(tour, Q, q, coords=xy)
    for K in (n, n + 3):
        fl = oracle.split_fleet(tour, Q, K, q, coords=xy)
        assert np.array_equal(fl["cost"], full["cost"])
    # every demand = Q: one route per customer, so K < n has no split
    qq = np.full((3, n), Q, np.int32)
    assert np.isinf(oracle.split_fleet(tour, Q, n - 1, qq, coords=xy)["cost"]).all()
    fl = oracle.split_fleet(tour, Q, n, qq, coords=xy)
    assert (fl["nroutes"] == n).all()
    np.testing.assert_allclose(fl["cost"], sum(euclid(xy, 0, c) + euclid(xy, c, 0) for c in tour),
                               rtol=1e-12)
    # n = 0
    e = oracle.split_fleet(np.zeros(0, np.int32), Q, 2, np.zeros((4, 0), np.int32),
                           coords=xy[:1])
    assert (e["cost"] == 0).all() and (e["nroutes"] == 0).all()


def test_fleet_monotone_in_K_and_routes_consistent():
    n, S, Q = 30, 60, 40
    tour, xy, q = _inst(11, n, S, Q, 12)
    prev = None
    for K in range(1, n + 1):
        o = oracle.split_fleet(tour, Q, K, q, coords=xy)
        if prev is not None:
            assert (o["cost"] <= prev + 1e-9 * np.abs(prev)).all()
        prev = np.where(np.isinf(o["cost"]), np.inf, o["cost"])
        fin = np.isfinite(o["cost"])
        assert (o["nroutes"][fin] <= K).all() and (o["nroutes"][~fin] == 0).all()
        for s in np.flatnonzero(fin)[:10]:
            r = o["route"][s]
            # routes numbered 0.. in tour order, contiguous, each within Q
            assert r[0] == 0 and (np.diff(r) >= 0).all() and (np.diff(r) <= 1).all()
            assert r[-1] + 1 == o["nroutes"][s]
            loads = np.bincount(r, weights=q[s][tour - 1])
            assert (loads <= Q).all()


def test_fleet_margin_is_positive_exactly_when_the_optimum_is_unique():
    """The margin is the tightest relative gap over the choices that make up
    the optimal split (the number of routes, then each route's start along
    the backtrack), so it certifies uniqueness.  With travel costs of 0, 1 or
    2 every sum is exact: margin > 0 if and only if brute force finds exactly
    one optimal split into at most K routes (+inf where none fits)."""
    unique = multiple = 0
    for seed in range(40):
        rng = np.random.default_rng(2900 + seed)
        n = int(rng.integers(2, 8))
        Q = int(rng.integers(2, 9))
        K = int(rng.integers(1, n + 1))
        d = rng.integers(0, 3, size=(n + 1, n + 1)).astype(np.float32)
        np.fill_diagonal(d, 0.0)
        tour = (rng.permutation(n) + 1).astype(np.int32)
        q = rng.integers(0, Q + 1, size=(4, n)).astype(np.int32)
        o = oracle.split_fleet(tour, Q, K, q, dist=d, want_margin=True)
        for s in range(4):
            best, parts = split_brute(tour.tolist(), q[s].tolist(), Q,
                                      lambda a, b: float(d[a, b]), max_routes=K)
            if math.isinf(best):
                assert math.isinf(o["margin"][s])
                continue
            assert (o["margin"][s] > 0) == (len(parts) == 1), (seed, s, parts)
            unique += len(parts) == 1
            multiple += len(parts) > 1
    assert unique >= 10 and multiple >= 10


@pytest.mark.parametrize("K", [2, 9])
def test_fleet_mean_is_the_sample_average(K):
    """The mean is the average of the per-scenario costs over all S (the SAA
    mean), +inf as soon as one scenario has no split into K routes."""
    tour, xy, q = _inst(7, 9, 50, 30, 12)
    o = oracle.split_fleet(tour, 30, K, q, coords=xy)
    c = o["cost"]
    if np.isinf(c).any():
        assert K == 2 and math.isinf(o["mean"])
    else:
        assert o["mean"] == pytest.approx(math.fsum(c) / len(c), rel=1e-14)

"""Pins of the route-option reinsertion oracle (an entry of the transition
matrix is a minimum over candidate routes; reading: route r on day t costs
rcost[t][r] and carries the delivery only if its residual capacity
cap[s][t][r] >= U - I) against brute force over every action sequence,
the two-action DP it generalises, and invariants."""
import math

import numpy as np
import pytest

import oracle
from tests import brute


def _case(rng, S, T, U, K, lam, cap_lo=0):
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    rcost = rng.uniform(5, 50, size=(T, K)).astype(np.float32)
    cap = rng.integers(cap_lo, U + 1, size=(S, T, K)).astype(np.int32)
    return cons, rcost, cap


@pytest.mark.parametrize("seed", range(30))
def test_routes_brute_force(seed):
    rng = np.random.default_rng(700 + seed)
    T = int(rng.integers(1, 6))
    U = int(rng.integers(0, 13))
    K = int(rng.integers(1, 4))
    I0 = int(rng.integers(0, U + 1))
    uc = float(rng.choice([0.0, 0.6]))
    cons, rcost, cap = _case(rng, 1, T, U, K, lam=float(rng.uniform(0.5, 6)))
    use_table = seed % 3 == 0
    H = rng.uniform(0, 9, U + 1) if use_table else None
    o = oracle.reinsert_routes(T, U, I0, 1.0, 7.0, uc, rcost, cap, cons, H=H)
    best, seqs = brute.reinsert_routes_brute(T, U, I0, 1.0, 7.0, uc, rcost, cap[0], cons[0], H=H)
    assert abs(o["value"][0] - best) <= 1e-12 * max(1.0, abs(best))
    if len(seqs) == 1:
        assert tuple(int(x) for x in o["policy"][0]) == seqs[0]


@pytest.mark.parametrize("seed", range(4))
def test_one_roomy_route_is_the_two_action_dp(seed):
    """K = 1 with a capacity of at least U every day: the route is always
    available and costs fixed[t], so values, C_0 tables and policies are
    those of the two-action DP."""
    rng = np.random.default_rng(800 + seed)
    S, T, U, I0 = 40, 20, 60, 30
    cons = rng.poisson(8.0, size=(S, T)).astype(np.int32)
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    cap = np.full((S, T, 1), U, np.int32)
    o1 = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, 0.3, fixed[:, None], cap, cons,
                                want_value0=True)
    o2 = oracle.reinsert(T, U, I0, 1.0, 20.0, 0.3, fixed, cons, want_value0=True)
    np.testing.assert_array_equal(o1["value"], o2["value"])
    np.testing.assert_array_equal(o1["value0"], o2["value0"])
    np.testing.assert_array_equal(o1["policy"], o2["policy"])


def test_no_room_means_no_delivery():
    """Every residual capacity 0: no delivery is ever possible, so the value
    is the simulated cost of never delivering."""
    rng = np.random.default_rng(9)
    S, T, U, I0, h, p = 30, 15, 40, 25, 1.0, 20.0
    cons = rng.poisson(6.0, size=(S, T)).astype(np.int32)
    rcost = rng.uniform(5, 50, (T, 3)).astype(np.float32)
    cap = np.zeros((S, T, 3), np.int32)
    o = oracle.reinsert_routes(T, U, I0, h, p, 0.0, rcost, cap, cons)
    assert not o["policy"].any()
    for s in range(S):
        I, v = I0, 0.0
        for t in range(T):
            x = I - int(cons[s, t])
            v += h * x if x >= 0 else p * (-x)
            I = max(0, x)
        assert abs(o["value"][s] - v) <= 1e-12 * max(1.0, v)


def test_more_routes_never_cost_more_and_ties_take_the_first():
    rng = np.random.default_rng(10)
    S, T, U, I0 = 50, 25, 80, 40
    cons, rcost, cap = _case(rng, S, T, U, 3, lam=10.0)
    prev = None
    for K in (1, 2, 3):
        v = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, 0.0, rcost[:, :K], cap[:, :, :K], cons)["value"]
        if prev is not None:
            assert np.all(v <= prev)
        prev = v
    # a duplicate of route 0 changes nothing, and the first copy is chosen
    r2 = np.concatenate([rcost[:, :1], rcost[:, :1]], axis=1)
    c2 = np.concatenate([cap[:, :, :1], cap[:, :, :1]], axis=2)
    a = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, 0.0, rcost[:, :1], cap[:, :, :1], cons)
    b = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, 0.0, r2, c2, cons)
    np.testing.assert_array_equal(a["value"], b["value"])
    np.testing.assert_array_equal(a["policy"], b["policy"])
    assert not math.isnan(float(b["mean"]))


@pytest.mark.parametrize("seed", range(12))
def test_routes_margin_by_brute_force(seed):
    """The margin at (t, I) equals (second - best) / max(|best|, |second|)
    over the values of every allowed action at (t, I) -- no delivery, or a
    route whose capacity holds U - I -- with every later day optimal, found
    by simulating every continuation; +inf where a single action exists."""
    rng = np.random.default_rng(760 + seed)
    T = int(rng.integers(1, 5))
    U = int(rng.integers(1, 8))
    K = int(rng.integers(1, 4))
    uc = float(rng.choice([0.0, 0.6]))
    cons, rcost, cap = _case(rng, 1, T, U, K, lam=float(rng.uniform(0.5, 5)))
    H = rng.uniform(0.5, 9, U + 1) if seed % 3 == 0 else None
    o = oracle.reinsert_routes(T, U, 0, 1.0, 7.0, uc, rcost, cap, cons, H=H, want_margin=True)
    mg = o["margin"][0]
    for t in range(T):
        for I in range(U + 1):
            v = brute.reinsert_action_values(T, U, 1.0, 7.0, uc, None, cons[0], t, I, H=H,
                                             rcost=rcost, cap=cap[0])
            vals = sorted(v.values())
            if len(vals) < 2:
                assert math.isinf(mg[t, I]), (t, I)
                continue
            den = max(abs(vals[0]), abs(vals[1]))
            expect = (vals[1] - vals[0]) / den if den > 0 else 0.0
            assert mg[t, I] == pytest.approx(expect, rel=1e-9, abs=1e-12), (t, I)

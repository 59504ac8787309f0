"""Pins of the reinsertion oracle (Algorithm SolveBatchDP, Eq. eqdp2) against
the paper's worked examples, brute-force enumeration of all delivery
sequences, closed forms and monotonicity."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests import brute
from tests.golden_io import arr, load


def test_minplus_toy():
    g = load("minplus_toy.json")
    out, arg = oracle.minplus_matvec(arr(g["A_t"]), arr(g["J_t"]))
    np.testing.assert_array_equal(out, arr(g["J_t1"]))
    np.testing.assert_array_equal(arg, arr(g["argmin"], np.int32))


def test_inventory_toy_forward_and_backward():
    g = load("inventory_toy.json")
    T, U, I0 = g["T"], g["U"], g["I0"]
    H = arr(g["end_cost_table"])
    fixed = np.zeros(T, np.float32)   # F_t(q) = q: no fixed part, unit cost 1
    cons = arr(g["consumption"], np.int32)
    v, Jh, A = oracle.reinsert_forward(T, U, I0, 0.0, 0.0, 1.0, fixed, cons, H=H, want_A=True)
    np.testing.assert_array_equal(A[0], arr(g["A1"]))
    np.testing.assert_array_equal(A[1], arr(g["A1"]))  # same parameters on day 2
    np.testing.assert_array_equal(Jh[0], arr(g["J1"]))
    np.testing.assert_array_equal(Jh[1], arr(g["J2"]))
    np.testing.assert_array_equal(Jh[2], arr(g["J3"]))
    assert v == g["value"]
    r = oracle.reinsert(T, U, I0, 0.0, 0.0, 1.0, fixed, cons[None, :], H=H)
    assert r["value"][0] == g["value"]
    np.testing.assert_array_equal(r["policy"][0], arr(g["policy"], np.uint8))


def _rand_params(rng, T, U):
    h = float(rng.uniform(0, 3))
    p = float(rng.uniform(0, 40))
    c = float(rng.choice([0.0, rng.uniform(0, 2)]))
    fixed = rng.uniform(0, 60, size=T).astype(np.float32)
    return h, p, c, fixed


@pytest.mark.parametrize("seed", range(40))
def test_reinsert_brute_force(seed):
    rng = np.random.default_rng(2000 + seed)
    T = int(rng.integers(1, 9))
    U = int(rng.integers(0, 13))
    I0 = int(rng.integers(0, U + 1))
    h, p, c, fixed = _rand_params(rng, T, U)
    H = rng.uniform(0, 20, size=U + 1) if seed % 4 == 3 else None
    cons = rng.integers(0, U + 3, size=T).astype(np.int32)
    best, seqs = brute.reinsert_brute(T, U, I0, h, p, c, fixed, cons, H=H)
    r = oracle.reinsert(T, U, I0, h, p, c, fixed, cons[None, :], H=H, want_value0=True)
    assert abs(r["value"][0] - best) <= 1e-12 * max(1.0, abs(best))
    assert r["value0"][0][I0] == r["value"][0]
    v, _, _ = oracle.reinsert_forward(T, U, I0, h, p, c, fixed, cons, H=H)
    assert abs(v - best) <= 1e-12 * max(1.0, abs(best))
    # the backtracked policy is one of the optimal sequences; when the optimum
    # is unique it is that sequence up to the no-op "deliver at I = U" choice
    pol = tuple(int(x) for x in r["policy"][0])
    def canon(seq):
        I, out = I0, []
        for t, a in enumerate(seq):
            a = a if I < U else 0
            out.append(a)
            I = max(0, I + ((U - I) if a else 0) - int(cons[t]))
        return tuple(out)
    assert canon(pol) in {canon(s) for s in seqs}


def test_reinsert_zero_consumption_never_delivers():
    T, U, I0 = 10, 20, 7
    fixed = np.full(T, 5.0, np.float32)
    cons = np.zeros((3, T), np.int32)
    r = oracle.reinsert(T, U, I0, 1.5, 20.0, 0.0, fixed, cons)
    np.testing.assert_allclose(r["value"], T * 1.5 * I0, rtol=1e-15)
    assert not r["policy"].any()


def test_reinsert_free_inventory_costs_nothing():
    T, U, I0 = 12, 30, 4
    fixed = np.linspace(5, 50, T).astype(np.float32)
    cons = np.random.default_rng(1).integers(0, 20, size=(4, T)).astype(np.int32)
    r = oracle.reinsert(T, U, I0, 0.0, 0.0, 0.0, fixed, cons)
    np.testing.assert_array_equal(r["value"], 0.0)
    assert not r["policy"].any()


def test_reinsert_deliver_every_day_closed_form():
    """Every d_t >= U and stockouts dearer than deliveries: deliver daily.
    Value = sum f_t + c((U - I0) + (T-1)U) + p sum (d_t - U)."""
    T, U, I0, h, p, c = 9, 15, 3, 1.0, 20.0, 0.5
    rng = np.random.default_rng(5)
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    cons = rng.integers(U, U + 10, size=(1, T)).astype(np.int32)
    assert (p - c) * (U - I0) > fixed.max()
    r = oracle.reinsert(T, U, I0, h, p, c, fixed, cons)
    expect = float(fixed.astype(np.float64).sum()) + c * ((U - I0) + (T - 1) * U) \
        + p * float((cons[0] - U).sum())
    assert r["value"][0] == pytest.approx(expect, rel=1e-14)
    assert r["policy"].all()


def test_reinsert_monotone_in_costs():
    spec = wl.REINSERT_C3
    cons = wl.reinsert_consumption(spec, 0, 50)[:, :20]
    T, U, I0 = 20, 60, 30
    fixed = wl.reinsert_fixed(spec)[:T]
    base = oracle.reinsert(T, U, I0, 1.0, 20.0, 0.0, fixed, cons)["value"]
    for kw in ({"h": 1.5}, {"p": 25.0}, {"c": 0.3}, {"f": 1.2}):
        h = kw.get("h", 1.0); p = kw.get("p", 20.0); c = kw.get("c", 0.0)
        f = (fixed * np.float32(kw.get("f", 1.0))).astype(np.float32)
        v = oracle.reinsert(T, U, I0, h, p, c, f, cons)["value"]
        assert np.all(v >= base - 1e-9)


def test_reinsert_forward_equals_backward_on_workload_sample():
    spec = wl.REINSERT_C3
    cons = wl.reinsert_consumption(spec, 0, 8)
    fixed = wl.reinsert_fixed(spec)
    r = oracle.reinsert(spec.T, spec.U, spec.I0, spec.h, spec.p, spec.unit_cost, fixed,
                        cons, want_value0=True)
    for s in range(cons.shape[0]):
        v, _, _ = oracle.reinsert_forward(spec.T, spec.U, spec.I0, spec.h, spec.p,
                                          spec.unit_cost, fixed, cons[s])
        assert v == pytest.approx(r["value"][s], rel=1e-12)
    assert np.all(np.isfinite(r["value0"]))
    assert abs(r["mean"] - r["value"].mean()) <= 1e-12 * r["mean"]


def test_reinsert_ties_prefer_no_delivery_by_brute_force():
    """Reading R6: with integer costs every action value is exact, so ties
    between delivering and not delivering are exact.  Along the oracle's
    path each day's decision must be to deliver exactly when delivering is
    strictly cheaper than not, both values with every later day optimal
    found by simulating every continuation."""
    ties = 0
    for seed in range(30):
        rng = np.random.default_rng(2800 + seed)
        T = int(rng.integers(1, 6))
        U = int(rng.integers(1, 6))
        h, p, c = float(rng.integers(0, 2)), float(rng.integers(0, 3)), float(rng.integers(0, 2))
        fixed = rng.integers(0, 3, size=T).astype(np.float32)
        cons = rng.integers(0, U + 2, size=T).astype(np.int32)
        I0 = int(rng.integers(0, U + 1))
        pol = oracle.reinsert(T, U, I0, h, p, c, fixed, cons[None, :])["policy"][0]
        I = I0
        for t in range(T):
            v = brute.reinsert_action_values(T, U, h, p, c, fixed, cons, t, I)
            if I == U:
                expect = 0
            else:
                ties += v[0] == v[1]
                expect = 1 if v[1] < v[0] else 0
            assert pol[t] == expect, (seed, t, I, v)
            I = max(0, (U if pol[t] else I) - int(cons[t]))
    assert ties >= 5


@pytest.mark.parametrize("seed", range(12))
def test_reinsert_margin_by_brute_force(seed):
    """The margin at (t, I) -- the relative gap between the two actions,
    which decides where the GPU's policy is compared bit for bit -- equals
    |v1 - v0| / max(|v0|, |v1|) for the values of delivering (v1) and not
    delivering (v0) at (t, I) with every later day optimal, both found by
    simulating every continuation; +inf where only one action exists (I = U)."""
    rng = np.random.default_rng(2600 + seed)
    T = int(rng.integers(1, 6))
    U = int(rng.integers(1, 9))
    h, p, c, fixed = _rand_params(rng, T, U)
    H = rng.uniform(0.5, 20, size=U + 1) if seed % 3 == 2 else None
    cons = rng.integers(0, U + 3, size=T).astype(np.int32)
    r = oracle.reinsert(T, U, 0, h, p, c, fixed, cons[None, :], H=H, want_margin=True)
    mg = r["margin"][0]
    for t in range(T):
        for I in range(U + 1):
            v = brute.reinsert_action_values(T, U, h, p, c, fixed, cons, t, I, H=H)
            if I == U:
                assert list(v) == [0] and math.isinf(mg[t, I])
                continue
            den = max(abs(v[0]), abs(v[1]))
            expect = abs(v[1] - v[0]) / den if den > 0 else 0.0
            assert mg[t, I] == pytest.approx(expect, rel=1e-9, abs=1e-12), (t, I)

"""GPU parity of the warp-per-scenario recomputation of flagged scenarios
(split_rescue.cu): when a deque kernel's ring cannot hold a scenario's deque,
the scenario is recomputed by one warp; its costs and predecessors must be
the plain kernel's bits and the oracle's values, through the C ABI."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import check_split

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _flat(n, S, Q, seed, qhi=2):
    """All travel costs zero: every candidate ties, nothing pops from the
    back, and with demands in {0..qhi} the windows (about Q / mean demand
    positions, often more than 32) outgrow every ring."""
    rng = np.random.default_rng(seed)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, qhi + 1, size=(S, n)).astype(np.int32)
    xy = np.full((n + 1, 2), 50.0, np.float32)
    return tour, xy, q


def _same(r, p):
    assert torch.equal(r["cost"], p["cost"])
    if r["pred"] is not None:
        assert torch.equal(r["pred"], p["pred"])


@pytest.mark.parametrize("algo", ["pipe", "stream", "deque"])
@pytest.mark.parametrize("preds", ["u16", "i32", None])
@pytest.mark.parametrize("n", [40, 301, 1000])
def test_rescue_matches_plain_on_ring_overflow(algo, preds, n):
    S, Q = 70, 40
    tour, xy, q = _flat(n, S, Q, seed=n)
    args = (_cuda(tour), Q, _cuda(q))
    sdp().status()
    r = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo=algo)
    st = sdp().status()
    p = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="plain")
    torch.cuda.synchronize()
    assert st & sdp().FLAG_FALLBACK
    _same(r, p)
    assert (r["cost"].cpu().numpy() == 0.0).all()


def test_rescue_windows_over_32_against_oracle():
    """Customers on a ray from the depot with sparse unit demands: psi rises
    along the tour, windows span 50+ positions (two or more chunks of 32
    candidates per step), and the optimum is unique: the recomputed scenarios
    match the oracle's costs and predecessors."""
    n, S, Q = 200, 64, 6
    xy = np.zeros((n + 1, 2), np.float32)
    xy[1:, 0] = np.arange(1, n + 1, dtype=np.float32) ** 1.25
    tour = np.arange(1, n + 1, dtype=np.int32)
    rng = np.random.default_rng(4)
    q = (rng.random((S, n)) < 0.1).astype(np.int32)
    orc = oracle.split(tour, Q, q, coords=xy, want_margin=True)
    for algo in ("pipe", "stream", "deque"):
        sdp().status()
        r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32", algo=algo)
        assert sdp().status() & sdp().FLAG_FALLBACK
        check_split(r["cost"], r["pred"], orc, min_checked=0.0)
        p = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32",
                             algo="plain")
        torch.cuda.synchronize()
        _same(r, p)


def test_rescue_infeasible_and_negative():
    """Flagged scenarios that also hold a demand above Q (cost +inf,
    predecessor -1 from that position on) or a negative demand (read as 0):
    the plain kernel's bits and both status flags."""
    n, S, Q = 120, 96, 30
    tour, xy, q = _flat(n, S, Q, seed=11)
    q[3, 50] = Q + 5
    q[40, 0] = Q + 1
    q[41, n - 1] = 10 * Q
    q[70, 17] = -4
    for algo in ("pipe", "stream", "deque"):
        for preds in ("u16", "i32"):
            sdp().status()
            r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds=preds,
                                 algo=algo)
            st = sdp().status()
            p = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds=preds,
                                 algo="plain")
            torch.cuda.synchronize()
            assert st & sdp().FLAG_FALLBACK and st & sdp().FLAG_INFEASIBLE
            assert st & sdp().FLAG_NEG_INPUT
            _same(r, p)
            c = r["cost"].cpu().numpy()
            assert np.isinf(c[[3, 40, 41]]).all() and np.isfinite(np.delete(c, [3, 40, 41])).all()


def test_rescue_long_tour_deep_deques():
    """A seeded n = 1000 tour with Q = 400 and demands U{1..30}: deques of
    13-16 entries occur (the PIPE ring test flags some scenarios); every
    path gives the same bits, whichever scenarios it recomputed."""
    n, S, Q = 1000, 8192, 400
    rng = np.random.default_rng(1000)
    xy = rng.uniform(0, 100, (n + 1, 2)).astype(np.float32)
    xy[0] = (50, 50)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 31, size=(S, n)).astype(np.int32)
    args = (_cuda(tour), Q, _cuda(q))
    ref = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo="stream")
    for algo in ("pipe", "deque"):
        r = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo=algo)
        torch.cuda.synchronize()
        _same(r, ref)
    rows = np.arange(0, S, 257)
    p = sdp().split_eval(_cuda(tour), Q, _cuda(q[rows]), coords=_cuda(xy), preds="u16",
                         algo="plain")
    torch.cuda.synchronize()
    assert torch.equal(ref["cost"][rows], p["cost"]) and torch.equal(ref["pred"][rows], p["pred"])
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("algo", ["pipe", "stream", "deque"])
def test_rescue_batched_plan(algo):
    """A batch whose even tours have zero travel costs (their scenarios all
    flag) and whose odd tours are ordinary: every cost is the one-tour plain
    kernel's bits."""
    B, S, Q = 6, 80, 25
    rng = np.random.default_rng(21)
    n = np.array([60, 9, 300, 33, 1, 130], np.int32)
    tours = [(rng.permutation(k) + 1).astype(np.int32) for k in n]
    coords = [np.full((k + 1, 2), 50.0, np.float32) if b % 2 == 0 else
              np.concatenate([[[50, 50]], rng.uniform(0, 100, (k, 2))]).astype(np.float32)
              for b, k in enumerate(n)]
    dem = [rng.integers(0, 3, size=(S, k)).astype(np.int32) for k in n]
    dem[2][7, 100] = Q + 1
    t = torch.from_numpy(np.concatenate(tours)).cuda()
    c = torch.from_numpy(np.concatenate(coords)).cuda()
    d = torch.from_numpy(np.concatenate([x.reshape(-1) for x in dem])).cuda()
    plan = sdp().SplitPlan(n, t, c, d, Q, S)
    plan.configure({"pipe": -2, "stream": -1, "deque": 4}[algo], 16, 1)
    sdp().status()
    costs, _ = plan.run()
    torch.cuda.synchronize()
    st = sdp().status()
    assert st & sdp().FLAG_FALLBACK and st & sdp().FLAG_INFEASIBLE
    for b in range(B):
        p = sdp().split_eval(_cuda(tours[b]), Q, _cuda(dem[b]), coords=_cuda(coords[b]),
                             algo="plain")
        torch.cuda.synchronize()
        assert torch.equal(costs[b], p["cost"]), b
    plan.close()

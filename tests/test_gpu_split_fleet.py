"""GPU parity of the fleet-limited Split (at most K routes; one warp per
scenario with the route counts across its lanes, and the one-thread-per-
scenario PLAIN kernel) against the FP64 oracle and each other, through the
C ABI."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.golden_io import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, MARGIN = 1e-5, 1e-4


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(seed, n, S, Q, qlo, qhi, dist_mode=False):
    rng = np.random.default_rng(seed)
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50, 50)
    xy[1:] = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(qlo, qhi + 1, size=(S, n)).astype(np.int32)
    dist = wl.dist_matrix_f32(xy) if dist_mode else None
    return tour, xy, dist, q


def _check(r, o, rows=None, margin=MARGIN):
    c = r["cost"].cpu().double().numpy()
    nr = r["nroutes"].cpu().numpy()
    ro = r["route"].cpu().numpy().astype(np.int64) if r["route"] is not None else None
    if rows is not None:
        c, nr = c[rows], nr[rows]
        ro = ro[rows] if ro is not None else None
    oc = o["cost"]
    assert np.array_equal(np.isinf(c), np.isinf(oc)), "infeasibility differs"
    fin = np.isfinite(oc)
    if fin.any():
        rel = np.abs(c[fin] - oc[fin]) / np.abs(oc[fin])
        assert rel.max() <= RTOL, rel.max()
    assert (nr[~fin] == 0).all()
    uniq = fin & (o["margin"] > margin)
    assert np.array_equal(nr[uniq], o["nroutes"][uniq])
    if ro is not None:
        assert (ro[~fin] == 255).all()
        assert np.array_equal(ro[uniq], o["route"][uniq])
    return uniq.mean() if len(uniq) else 1.0


def test_fleet_paper_example():
    """Tour (1,2,4,3,5), Q = 17: the scenarios that need 3 and 2 routes are
    infeasible below that fleet and feasible at it; with three vehicles the
    split uses at least the minimum and at most three routes."""
    g = load("split_figure_feasibility.json")
    tour = np.asarray(g["tour"], np.int32)
    rng = np.random.default_rng(3)
    xy = rng.uniform(0, 100, (len(tour) + 1, 2)).astype(np.float32)
    q = np.asarray([sc["demand_by_customer"] for sc in g["scenarios"]], np.int32)
    mins = [sc["min_routes"] for sc in g["scenarios"]]
    for K in (1, 2, 3, 4):
        r = sdp().split_fleet_eval(_cuda(tour), g["Q"], _cuda(q), K, coords=_cuda(xy))
        o = oracle.split_fleet(tour, g["Q"], K, q, coords=xy, want_margin=True)
        torch.cuda.synchronize()
        _check(r, o)
        nr = r["nroutes"].cpu().numpy()
        for s, m in enumerate(mins):
            assert (nr[s] == 0) == (K < m)
            if K == 3:
                assert m <= nr[s] <= 3
    sdp().status()


@pytest.mark.parametrize("case", [
    # seed, n, S, Q, qlo, qhi, K, dist
    (1, 8, 70, 30, 1, 15, 3, False),
    (2, 40, 100, 60, 1, 20, 12, False),
    (3, 37, 65, 40, 0, 45, 20, True),     # zero demands, some demand > Q, dist mode
    (4, 100, 64, 100, 1, 30, 33, False),  # two slots per lane
    (5, 150, 40, 150, 5, 25, 30, False),  # K near the minimum number of routes
    (6, 1, 33, 10, 1, 12, 1, False),      # n = 1
    (7, 60, 50, 300, 1, 40, 64, False),   # uint16-range Q, the largest K
])
def test_fleet_cases_vs_oracle_and_plain(case):
    seed, n, S, Q, qlo, qhi, K, dm = case
    tour, xy, dist, q = _case(seed, n, S, Q, qlo, qhi, dm)
    kw = {"dist": dist} if dm else {"coords": xy}
    o = oracle.split_fleet(tour, Q, K, q, want_margin=True, **kw)
    args = (_cuda(tour), Q, _cuda(q), K)
    ck = {k: _cuda(v) for k, v in kw.items()}
    r = sdp().split_fleet_eval(*args, **ck)
    p = sdp().split_fleet_eval(*args, algo="plain", **ck)
    torch.cuda.synchronize()
    _check(r, o)
    _check(p, o)
    for key in ("cost", "nroutes", "route"):
        assert torch.equal(r[key], p[key]), key
    if np.isinf(o["cost"]).any():
        assert sdp().status() & sdp().FLAG_INFEASIBLE
    else:
        assert abs(float(r["mean"]) - o["mean"]) <= RTOL * abs(o["mean"])
        assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("n", [5, 31, 60])
def test_fleet_without_a_binding_limit_is_split(n):
    """K >= n: every layer is allowed, and the minimum over the layers is the
    Split recursion's own minimum, FP32 operation for operation."""
    tour, xy, _, q = _case(50 + n, n, 200, 50, 1, 20)
    args = (_cuda(tour), 50, _cuda(q))
    r = sdp().split_fleet_eval(*args, min(64, max(n, 1)), coords=_cuda(xy), routes=False)
    s = sdp().split_eval(*args, coords=_cuda(xy), preds="i32", algo="deque")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], s["cost"])
    # the route count of the unlimited split, where its predecessors are unique
    o = oracle.split(tour, 50, q, coords=xy, want_margin=True)
    nr = r["nroutes"].cpu().numpy()
    for sc in range(q.shape[0]):
        if (o["margin"][sc] > MARGIN).all():
            i, k = n, 0
            while i > 0:
                i = o["pred"][sc][i - 1]
                k += 1
            assert nr[sc] == k


def test_fleet_ring_overflow_fallback():
    """All travel costs zero: every candidate ties and stays in the deque, so
    windows longer than the ring send those scenarios to the plain kernel."""
    n, S, Q, K = 40, 70, 40, 6
    rng = np.random.default_rng(9)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, 3, size=(S, n)).astype(np.int32)
    xy = np.full((n + 1, 2), 50.0, np.float32)
    r = sdp().split_fleet_eval(_cuda(tour), Q, _cuda(q), K, coords=_cuda(xy))
    p = sdp().split_fleet_eval(_cuda(tour), Q, _cuda(q), K, coords=_cuda(xy), algo="plain")
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    for key in ("cost", "nroutes", "route"):
        assert torch.equal(r[key], p[key]), key
    assert (r["cost"].cpu().numpy() == 0.0).all()
    # every split costs 0: the fewest routes, which packing the tour greedily
    # into consecutive routes of load <= Q gives
    o = oracle.split_fleet(tour, Q, K, q, coords=xy)
    greedy = []
    for row in q[:, tour - 1]:
        k, load = 1, 0
        for d in row:
            if load + d > Q:
                k, load = k + 1, 0
            load += d
        greedy.append(k)
    assert np.array_equal(r["nroutes"].cpu().numpy(), o["nroutes"])
    assert np.array_equal(o["nroutes"], np.asarray(greedy))


def test_fleet_bench_shape_sampled():
    """n = 500, Q = 200, demands U{1..30} (the Split benchmark's recipe), fleet
    K = 42: the limit binds (the sampled feasible scenarios use all 42 routes,
    about a tenth need more); sampled scenarios against the oracle (routes
    compared where the optimum is unique by 1e-5, as for the full-size Split),
    and the fleet never cheaper than the unlimited split."""
    spec = wl.SPLIT_C2
    tour, xy, _ = wl.split_tour(spec)
    S, K = 4096, 42
    q = wl.split_demands(spec, 0, S)
    r = sdp().split_fleet_eval(_cuda(tour), spec.Q, _cuda(q), K, coords=_cuda(xy))
    s = sdp().split_eval(_cuda(tour), spec.Q, _cuda(q), coords=_cuda(xy))
    torch.cuda.synchronize()
    rng = np.random.default_rng(2)
    rows = np.sort(rng.choice(S, 64, replace=False))
    o = oracle.split_fleet(tour, spec.Q, K, q[rows], coords=xy, want_margin=True)
    frac = _check(r, o, rows=rows, margin=1e-5)
    assert frac > 0.3
    c, u = r["cost"].cpu().numpy(), s["cost"].cpu().numpy()
    fin = np.isfinite(c)
    assert fin.mean() > 0.5 and (c[fin] >= u[fin] * (1 - 1e-6)).all()
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


def test_fleet_rejects():
    api = sdp()
    tour, xy, _, q = _case(1, 10, 8, 30, 1, 10)
    args = (_cuda(tour), 30, _cuda(q))
    for K in (0, 65):
        with pytest.raises(api.SdpError) as e:
            api.split_fleet_eval(*args, K, coords=_cuda(xy))
        assert e.value.code == -5
    with pytest.raises(api.SdpError) as e:
        api.split_fleet_eval(*args, 3, coords=_cuda(xy), algo="deque")
    assert e.value.code == -5

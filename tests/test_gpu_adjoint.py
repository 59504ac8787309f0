"""GPU parity of the Split adjoint (d mean / d dist = scenario-averaged
arc-usage counts of the optimal splits) through the C ABI and the autograd
binding: the fused forward + on-chip backtrack and the backtrack of stored
predecessors against the FP64 oracle's backtrack."""
import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.gpu_util import check_split, preds_to_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(seed, n, S, Q, lam):
    spec = wl.SplitSpec(f"adj{seed}", n, Q, S, seed, "poisson", lam=lam, lo=1, hi=Q,
                        dist_mode=True)
    tour, _, dist = wl.split_tour(spec)
    return tour, dist, wl.split_demands(spec)


def _gpu_preds(tour, Q, q, dist):
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), dist=_cuda(dist), preds="i32")
    torch.cuda.synchronize()
    return r, preds_to_i64(r["pred"]).astype(np.int32)


@pytest.mark.parametrize("case", [(1, 17, 70, 40, 8.0), (2, 60, 500, 80, 10.0),
                                  (3, 300, 2000, 120, 10.0), (4, 513, 96, 150, 12.0)])
@pytest.mark.parametrize("mode", ["fused", "pred_u16", "pred_i32"])
def test_adjoint_vs_oracle_backtrack(case, mode):
    seed, n, S, Q, lam = case
    tour, dist, q = _case(seed, n, S, Q, lam)
    orc = oracle.split(tour, Q, q, dist=dist, want_margin=True)
    r, gp = _gpu_preds(tour, Q, q, dist)
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)   # preds = oracle's where unique
    # the oracle's backtrack of the GPU's own optimal splits: exact counts
    g_ref = oracle.split_mean_grad(tour, gp)
    start, end, skipped = oracle.split_route_counts(gp)
    assert skipped == 0
    gm = torch.tensor(1.0, device="cuda")
    if mode == "fused":
        g, hist = sdp().split_backward(_cuda(tour), Q, _cuda(q), _cuda(dist), gm, want_hist=True)
    else:
        dt = mode.split("_")[1]
        p = sdp().split_eval(_cuda(tour), Q, _cuda(q), dist=_cuda(dist), preds=dt)["pred"]
        g, hist = sdp().split_backward(_cuda(tour), Q, _cuda(q), _cuda(dist), gm, pred=p,
                                       pred_dtype=dt, want_hist=True)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    np.testing.assert_array_equal(h[:n], start)
    np.testing.assert_array_equal(h[n:], end)
    np.testing.assert_allclose(g.cpu().double().numpy(), g_ref, rtol=1e-6, atol=1e-9)
    # against the oracle's own splits: only scenarios with a near-tie may differ
    g_orc = oracle.split_mean_grad(tour, orc["pred"])
    differ = int((gp != orc["pred"]).any(axis=1).sum())
    assert np.abs(g.cpu().double().numpy() - g_orc).max() <= 2.0 * differ / S + 1e-6


def test_adjoint_autograd_and_upstream_gradient():
    """SplitMeanCost.backward (stored predecessors and fused) equals the C ABI
    call, scaled by the upstream gradient."""
    tour, dist, q = _case(5, 80, 400, 60, 9.0)
    d = _cuda(dist).requires_grad_(True)
    t, qd = _cuda(tour), _cuda(q)
    for keep in (False, True):
        d.grad = None
        m = sdp().SplitMeanCost.apply(d, t, qd, 60, keep)
        (3.0 * m).backward()
        g, _ = sdp().split_backward(t, 60, qd, d.detach(), torch.tensor(3.0, device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(d.grad, g)
    r = sdp().split_eval(t, 60, qd, dist=d.detach())
    assert abs(float(m.detach()) - float(r["mean"])) == 0.0


def test_adjoint_skips_infeasible_scenarios():
    """A scenario with a demand above Q is infeasible (cost +inf) and
    contributes no arc; the others are averaged over all S."""
    tour, dist, q = _case(6, 40, 200, 50, 8.0)
    q[3, 5] = 51
    q[77, 0] = 999
    r, gp = _gpu_preds(tour, 50, q, dist)
    assert np.isinf(r["cost"][3].item()) and np.isinf(r["cost"][77].item())
    g_ref = oracle.split_mean_grad(tour, gp)
    g, hist = sdp().split_backward(_cuda(tour), 50, _cuda(q), _cuda(dist),
                                   torch.tensor(1.0, device="cuda"), want_hist=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(g.cpu().double().numpy(), g_ref, rtol=1e-6, atol=1e-9)
    start, _, skipped = oracle.split_route_counts(gp)
    assert skipped == 2
    np.testing.assert_array_equal(hist.cpu().numpy()[:40], start)
    sdp().status()


def test_adjoint_full_size():
    """n=300, S=10^5 (the adjoint workload) with the fused kernel: counts equal
    the oracle's backtrack of the GPU's predecessors."""
    spec = wl.ADJOINT_C5
    tour, _, dist = wl.split_tour(spec)
    qd = wl.split_demands_device(spec)
    t, dd = _cuda(tour), _cuda(dist)
    r = sdp().split_eval(t, spec.Q, qd, dist=dd, preds="i32")
    g, hist = sdp().split_backward(t, spec.Q, qd, dd, torch.tensor(1.0, device="cuda"),
                                   want_hist=True)
    torch.cuda.synchronize()
    gp = preds_to_i64(r["pred"]).astype(np.int32)
    start, end, skipped = oracle.split_route_counts(gp)
    assert skipped == 0
    h = hist.cpu().numpy()
    np.testing.assert_array_equal(h[:spec.n], start)
    np.testing.assert_array_equal(h[spec.n:], end)
    np.testing.assert_allclose(g.cpu().double().numpy(), oracle.split_mean_grad(tour, gp),
                               rtol=1e-6, atol=1e-9)
    rows = np.random.default_rng(4).choice(spec.S, 500, replace=False)
    qs = np.concatenate([wl.split_demands(spec, int(s), int(s) + 1) for s in rows])
    orc = oracle.split(tour, spec.Q, qs, dist=dist, want_margin=True)
    check_split(r["cost"], r["pred"], orc, rows=rows, margin=1e-5, min_checked=0.5)


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("case", [
    # (seed, n, Q, tiles per SM): the TMEM adjoint takes 16 warps per SM,
    # 17..24 when that many (as the row fits) finish every tile in one round
    (7, 17, 40, 0.5),      # n % 4 = 1, under one round
    (8, 300, 120, 20.6),   # 21 warps, one round
    (9, 300, 120, 24.0),   # 24 warps, exactly one round
    (10, 350, 120, 18.0),  # 88-word rows: at most 20 warps
    (11, 200, 300, 19.5),  # uint16 rows (Q >= 255), 100 words
    (12, 450, 150, 17.0),  # 113-word rows: 16 warps, two rounds
    (13, 301, 120, 49.3),  # beyond one round of 24: 16 warps, four rounds
])
def test_adjoint_tmem_equals_shared_staging(case):
    """The TMEM adjoint (default shape) and the shared-memory one (4 warps
    per CTA) take the same DP steps: identical counts, identical gradient,
    and both equal to the oracle's backtrack of the GPU's predecessors."""
    seed, n, Q, tps = case
    S = max(1, int(tps * _sms() * 32) - 5)   # a ragged last tile
    tour, dist, q = _case(seed, n, S, Q, 10.0 if Q < 255 else 25.0)
    t, qd, dd = _cuda(tour), _cuda(q), _cuda(dist)
    gm = torch.tensor(1.0, device="cuda")
    g0, h0 = sdp().split_backward(t, Q, qd, dd, gm, want_hist=True)
    g1, h1 = sdp().split_backward(t, Q, qd, dd, gm, want_hist=True, warps=4)
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK == 0
    assert torch.equal(h0, h1)
    assert torch.equal(g0, g1)
    assert int(h0[:n].sum()) >= S  # every scenario has at least one route
    if S <= 60000:
        r, gp = _gpu_preds(tour, Q, q, dist)
        start, end, skipped = oracle.split_route_counts(gp)
        assert skipped == 0
        h = h0.cpu().numpy()
        np.testing.assert_array_equal(h[:n], start)
        np.testing.assert_array_equal(h[n:], end)


def test_adjoint_tmem_route_longer_than_255_falls_back():
    """uint8 deltas hold routes of at most 255 customers: with zero demands a
    route may be longer, and such scenarios are recomputed (with their
    backtrack) by the plain kernel.  Counts equal the oracle's backtrack."""
    rng = np.random.default_rng(14)
    n, S, Q = 400, 200, 60
    spec = wl.SplitSpec("adj_zero", n, Q, S, 14, "poisson", lam=1.0, lo=1, hi=Q, dist_mode=True)
    tour, _, dist = wl.split_tour(spec)
    q = (rng.random((S, n)) < 0.05).astype(np.int32) * rng.integers(1, 30, (S, n)).astype(np.int32)
    q[:100] = 0                   # one route of all 400 customers
    q[100:105, 200] = Q           # a full customer splits it into three
    orc = oracle.split(tour, Q, q, dist=dist, want_margin=True)
    r, gp = _gpu_preds(tour, Q, q, dist)
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)
    g, hist = sdp().split_backward(_cuda(tour), Q, _cuda(q), _cuda(dist),
                                   torch.tensor(1.0, device="cuda"), want_hist=True)
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    start, end, skipped = oracle.split_route_counts(gp)
    assert skipped == 0
    h = hist.cpu().numpy()
    np.testing.assert_array_equal(h[:n], start)
    np.testing.assert_array_equal(h[n:], end)
    np.testing.assert_allclose(g.cpu().double().numpy(), oracle.split_mean_grad(tour, gp),
                               rtol=1e-6, atol=1e-9)


def test_adjoint_tmem_uint16_rows_with_over_capacity_demands():
    """Q >= 255 stages uint16 rows; demands above Q make their scenarios
    infeasible (no arc counted).  The TMEM adjoint, the shared-memory one and
    the oracle's backtrack of the GPU's predecessors agree."""
    n, S, Q = 180, 3000, 400
    tour, dist, q = _case(15, n, S, Q, 40.0)
    q[7, 3] = Q + 1
    q[2999, 179] = 5000
    t, qd, dd = _cuda(tour), _cuda(q), _cuda(dist)
    gm = torch.tensor(1.0, device="cuda")
    g0, h0 = sdp().split_backward(t, Q, qd, dd, gm, want_hist=True)
    g1, h1 = sdp().split_backward(t, Q, qd, dd, gm, want_hist=True, warps=4)
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_INFEASIBLE
    assert torch.equal(h0, h1) and torch.equal(g0, g1)
    r, gp = _gpu_preds(tour, Q, q, dist)
    start, end, skipped = oracle.split_route_counts(gp)
    assert skipped == 2
    h = h0.cpu().numpy()
    np.testing.assert_array_equal(h[:n], start)
    np.testing.assert_array_equal(h[n:], end)
    sdp().status()  # the forward above flags the same infeasible scenarios


def _path_positions(pred, n):
    """Positions i visited by the backtrack from n (where pred(i) decides the
    routes), per scenario."""
    out = []
    for row in pred:
        i, pos = n, []
        while i > 0:
            pos.append(i)
            i = int(row[i - 1])
        out.append(pos)
    return out


def _tie_free(orc, n, margin=1e-4):
    """Scenarios whose optimal routes are unique by more than `margin`
    relative at every position the oracle's backtrack visits."""
    keep = []
    for s, pos in enumerate(_path_positions(orc["pred"], n)):
        if all(orc["margin"][s, i - 1] > margin for i in pos):
            keep.append(s)
    return np.asarray(keep, np.int64)


@pytest.mark.parametrize("case", [(24, 40, 4000, 60, 1e-4), (23, 300, 3000, 120, 1e-6)])
@pytest.mark.parametrize("mode", ["fused", "pred_u16"])
def test_adjoint_equals_oracle_splits_where_tie_free(case, mode):
    """On the scenarios whose optimal routes are unique by more than `margin`
    relative along the oracle's backtrack, the GPU adjoint's route start /
    end counts equal those of the oracle's OWN optimal splits exactly, and
    its gradient equals the oracle's arc-usage gradient to FP32 rounding.
    1e-4 is the uniqueness the predecessor parity uses; at n = 300 no
    scenario is unique by 1e-4 at every visited position (J(i) reaches 10^4,
    so 1e-4 relative is about one distance unit), so that case takes 1e-6."""
    seed, n, S, Q, margin = case
    tour, dist, q = _case(seed, n, S, Q, 10.0)
    orc = oracle.split(tour, Q, q, dist=dist, want_margin=True)
    keep = _tie_free(orc, n, margin)
    assert keep.size >= S // 2
    qs = np.ascontiguousarray(q[keep])
    op = np.ascontiguousarray(orc["pred"][keep])
    start, end, skipped = oracle.split_route_counts(op)
    assert skipped == 0
    t, qd, dd = _cuda(tour), _cuda(qs), _cuda(dist)
    gm = torch.tensor(1.0, device="cuda")
    if mode == "fused":
        g, hist = sdp().split_backward(t, Q, qd, dd, gm, want_hist=True)
    else:
        p = sdp().split_eval(t, Q, qd, dist=dd, preds="u16")["pred"]
        g, hist = sdp().split_backward(t, Q, qd, dd, gm, pred=p, pred_dtype="u16",
                                       want_hist=True)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    np.testing.assert_array_equal(h[:n], start)
    np.testing.assert_array_equal(h[n:], end)
    np.testing.assert_allclose(g.cpu().double().numpy(), oracle.split_mean_grad(tour, op),
                               rtol=1e-6, atol=1e-9)


def test_adjoint_equals_central_differences_of_the_oracle_mean():
    """The GPU gradient (SplitMeanCost.backward) equals the central finite
    difference, h = 1e-3 in FP32, of the FP64 oracle's scenario mean at every
    checked entry of dist: the 3n structurally nonzero ones and 40 random
    zero ones, where every scenario's optimal routes at +h and -h are those
    at 0 (the mean is piecewise linear in dist, so the difference is exact
    there up to rounding).  Scenarios are those whose optimal routes are
    unique by more than 1e-4 relative, so the GPU's splits are the oracle's."""
    n, S, Q = 60, 2000, 80
    tour, dist, q = _case(22, n, S, Q, 10.0)
    orc = oracle.split(tour, Q, q, dist=dist, want_margin=True)
    keep = _tie_free(orc, n)
    assert keep.size >= S // 8
    q = np.ascontiguousarray(q[keep])
    base = oracle.split(tour, Q, q, dist=dist)
    routes0 = _path_positions(base["pred"], n)
    d = _cuda(dist).requires_grad_(True)
    m = sdp().SplitMeanCost.apply(d, _cuda(tour), _cuda(q), Q)
    m.backward()
    torch.cuda.synchronize()
    g = d.grad.cpu().double().numpy()
    assert abs(float(m.detach()) - base["mean"]) <= 1e-5 * abs(base["mean"])
    rng = np.random.default_rng(22)
    entries = [(0, int(c)) for c in tour] + [(int(c), 0) for c in tour]
    entries += [(int(a), int(b)) for a, b in zip(tour[:-1], tour[1:])]
    entries += [tuple(int(v) for v in rng.integers(1, n + 1, 2)) for _ in range(40)]
    h = np.float32(1e-3)
    checked = 0
    for (a, b) in entries:
        dp = dist.copy(); dp[a, b] += h
        dm = dist.copy(); dm[a, b] -= h
        rp = oracle.split(tour, Q, q, dist=dp)
        rm = oracle.split(tour, Q, q, dist=dm)
        if not (_path_positions(rp["pred"], n) == routes0 and
                _path_positions(rm["pred"], n) == routes0):
            continue  # a tie within h: the gradient is not defined there
        step = float(dp[a, b]) - float(dm[a, b])  # the FP32 perturbation applied
        fd = (rp["mean"] - rm["mean"]) / step
        assert g[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-7), (a, b)
        checked += 1
    assert checked >= 0.9 * len(entries)


@pytest.mark.parametrize("n,S", [(60, 3000), (300, 20000)])
def test_graphed_backward_replays_the_eager_bits(n, S):
    """GraphedSplitBackward (the fused adjoint step captured in a CUDA graph):
    every replay gives the eager call's gradient and route counts bit for
    bit; after the demands are refilled in place a replay gives the eager
    result for the new demands; and the gradient scales exactly with
    grad_mean (a factor of 4 is a power of two)."""
    tour, dist, q1 = _case(40 + n, n, S, 100, 9.0)
    _, _, q2 = _case(41 + n, n, S, 100, 9.0)
    t, d, q = _cuda(tour), _cuda(dist), _cuda(q1).clone()
    gm = torch.tensor(0.5, dtype=torch.float32, device="cuda")
    g = sdp().GraphedSplitBackward(t, 100, q, d, gm, want_hist=True)
    eg, eh = sdp().split_backward(t, 100, q, d, gm, want_hist=True)
    for _ in range(3):
        gg, gh = g.run()
        torch.cuda.synchronize()
        assert torch.equal(gg, eg) and torch.equal(gh, eh)
    q.copy_(_cuda(q2))
    eg2, eh2 = sdp().split_backward(t, 100, q, d, gm, want_hist=True)
    gg, gh = g.run()
    torch.cuda.synchronize()
    assert torch.equal(gg, eg2) and torch.equal(gh, eh2) and not torch.equal(eh2, eh)
    gm.fill_(2.0)
    gg, _ = g.run()
    torch.cuda.synchronize()
    assert torch.equal(gg, eg2 * 4)
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0

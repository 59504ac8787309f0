"""GPU parity of the SAA candidate search (current tour + B neighbours per
iteration, one batched-plan replay, best strict improvement taken) against
the oracle, which rebuilds the same moves from the SplitMix64 stream with list
operations and scores every candidate with the FP64 Split."""
import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative: FP32 route costs, FP64 means


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _instance(seed, n, S, Q, lam):
    rng = np.random.default_rng(seed)
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50, 50)
    xy[1:] = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    q = np.clip(rng.poisson(lam, (S, n)), 1, Q).astype(np.int32)
    tour0 = (rng.permutation(n) + 1).astype(np.int32)
    return tour0, xy, q


def _compare_trajectory(g_trace, g_acc, orc):
    """Iteration by iteration while the oracle's choice is unique by more
    than TOL: every neighbour scoring within TOL of the best is the same tour
    as the best (different moves can give one tour; both sides then take the
    first index), and the best is not within TOL of the current tour's score
    (reversing the whole tour keeps the mean, up to rounding).  Returns the
    number of iterations compared."""
    for t in range(len(orc["trace"])):
        ms = orc["means"][t]
        m0, nb = ms[0], ms[1:]
        kb = int(np.argmin(nb))
        near = np.nonzero(nb <= nb[kb] + TOL * abs(nb[kb]))[0]
        cands = orc["cands"][t]
        if any(not np.array_equal(cands[k], cands[kb]) for k in near):
            return t
        if abs(nb[kb] - m0) <= TOL * abs(m0):
            return t
        assert g_acc[t] == orc["accepted"][t], t
        assert abs(g_trace[t] - orc["trace"][t]) <= TOL * abs(orc["trace"][t]), t
    return len(orc["trace"])


@pytest.mark.parametrize("case", [
    # seed, n, S, Q, lam, B, iters, kinds, iterations that must compare
    (1, 20, 64, 40, 8.0, 32, 6, ("2opt", "relocate", "swap"), 1),
    (2, 37, 100, 60, 10.0, 96, 4, ("2opt",), 1),
    (3, 12, 33, 25, 6.0, 300, 3, ("relocate", "swap"), 1),
    (4, 2, 10, 9, 3.0, 5, 3, ("swap",), 0),  # n = 2: the one neighbour is the reversal
    (5, 150, 40, 100, 10.0, 64, 2, ("2opt", "relocate", "swap"), 1),
])
def test_search_vs_oracle(case):
    seed, n, S, Q, lam, B, iters, kinds, min_done = case
    tour0, xy, q = _instance(seed, n, S, Q, lam)
    orc = oracle.saa_search(tour0, Q, q, xy, B=B, iters=iters, seed=1000 + seed, kinds=kinds)
    s = sdp().SaaSearch(_cuda(tour0), _cuda(xy), _cuda(q), Q, B, seed=1000 + seed, moves=kinds)
    trace, acc = s.run(iters)
    tour, means = s.state()
    torch.cuda.synchronize()
    done = _compare_trajectory(trace.cpu().numpy(), acc.cpu().numpy(), orc)
    assert done >= min_done
    if done == iters:
        np.testing.assert_array_equal(tour.cpu().numpy(), orc["tour"])
        np.testing.assert_allclose(means.cpu().numpy(), orc["means"][-1], rtol=TOL)
    assert np.all(np.diff(trace.cpu().numpy()) <= 0)
    s.close()


def test_first_iteration_candidates_all_match():
    """All B + 1 scores of one iteration (the start tour and every neighbour,
    all three move kinds) against the oracle's scores of its own candidates."""
    tour0, xy, q = _instance(6, 45, 80, 50, 9.0)
    B = 700
    orc = oracle.saa_search(tour0, 50, q, xy, B=B, iters=1, seed=11)
    s = sdp().SaaSearch(_cuda(tour0), _cuda(xy), _cuda(q), 50, B, seed=11)
    s.run(1)
    _, means = s.state()
    torch.cuda.synchronize()
    np.testing.assert_allclose(means.cpu().numpy(), orc["means"][0], rtol=TOL)


def test_runs_continue_the_move_stream():
    tour0, xy, q = _instance(7, 30, 50, 40, 8.0)
    args = (_cuda(tour0), _cuda(xy), _cuda(q), 40, 40)
    a = sdp().SaaSearch(*args, seed=5)
    ta, aa = a.run(5)
    b = sdp().SaaSearch(*args, seed=5)
    tb1, ab1 = b.run(3)
    tb2, ab2 = b.run(2)
    torch.cuda.synchronize()
    assert torch.equal(ta, torch.cat([tb1, tb2])) and torch.equal(aa, torch.cat([ab1, ab2]))
    assert torch.equal(a.state()[0], b.state()[0])


def test_rejections():
    api = sdp()
    tour0, xy, q = _instance(8, 10, 20, 30, 5.0)
    t, c, d = _cuda(tour0), _cuda(xy), _cuda(q)
    for kw, code in ((dict(B=0), -1), (dict(moves=()), -1)):
        B = kw.pop("B", 8)
        with pytest.raises(api.SdpError) as e:
            api.SaaSearch(t, c, d, 30, B, **kw)
        assert e.value.code == code
    with pytest.raises(api.SdpError) as e:
        api.SaaSearch(t[:1].contiguous(), c[:2].contiguous(), d[:, :1].contiguous(), 30, 4)
    assert e.value.code == -5  # n = 1: no move exists


def test_search_workload_sampled():
    """n = 100, S = 10^4, 1024 neighbours (the search workload), two
    iterations: 40 sampled neighbour scores of the last iteration and the
    start tour's against the oracle; the trace is the minimum of the scores."""
    spec = wl.SAA_C6
    tour0, xy, _ = wl.split_tour(spec)
    qd = wl.split_demands_device(spec)
    s = sdp().SaaSearch(_cuda(tour0), _cuda(xy), qd, spec.Q, wl.SAA_B, seed=6)
    trace, acc = s.run(2)
    tour, means = s.state()
    torch.cuda.synchronize()
    m = means.cpu().numpy()
    tr, ac = trace.cpu().numpy(), acc.cpu().numpy()
    assert tr[1] == (m[1 + ac[1]] if ac[1] >= 0 else m[0])
    assert tr[1] == min(m[0], m[1:].min())
    q = wl.split_demands(spec)
    # rebuild iteration 1's start tour and candidates with the oracle's moves
    x0 = list(tour0)
    if ac[0] >= 0:
        x0 = oracle.apply_move(x0, *oracle.draw_move(6, int(ac[0]), spec.n))
    rng = np.random.default_rng(0)
    for k in [-1] + list(rng.choice(wl.SAA_B, 40, replace=False)):
        cand = x0 if k < 0 else oracle.apply_move(x0, *oracle.draw_move(6, wl.SAA_B + int(k),
                                                                        spec.n))
        ref = oracle.split(np.asarray(cand, np.int32), spec.Q, q, coords=xy,
                           want_pred=False)["mean"]
        assert abs(m[1 + k] - ref) <= TOL * ref, k
    s.close()


def test_autotune_keeps_the_trajectory(tmp_path):
    """Every launch shape computes the same costs: an autotuned search takes
    the same steps as one on the default shape, bit for bit."""
    tour0, xy, q = _instance(9, 60, 300, 50, 7.0)
    args = (_cuda(tour0), _cuda(xy), _cuda(q), 50, 128)
    a = sdp().SaaSearch(*args, seed=21)
    b = sdp().SaaSearch(*args, seed=21)
    shape = b.autotune(str(tmp_path / "cache.txt"))
    # the search's plan reports the shape the autotune chose (deque rings of
    # 16 entries only, or one of the producer/consumer kernels)
    assert shape == b.info() and shape["ring"] == 16
    assert shape["warps_per_cta"] in (-2, -1, 0, 1, 2, 4, 8) and shape["scenarios_per_lane"] in (1, 2)
    sdp().status()
    ta, aa = a.run(6)
    tb, ab = b.run(6)
    torch.cuda.synchronize()
    assert torch.equal(ta, tb) and torch.equal(aa, ab)
    assert sdp().status() & sdp().FLAG_FALLBACK == 0

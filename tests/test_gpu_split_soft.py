"""GPU parity of the soft-capacity Split (every split allowed, a penalty per
unit of route load above Q) against the FP64 oracle, through the C ABI:
PLAIN relaxes every pair (p, i); DEQUE keeps the hard window in its deque
and the expired entries as one running minimum."""
import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.gpu_util import check_split

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(seed, n, S, qlo, qhi, dist_mode=False):
    rng = np.random.default_rng(seed)
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50, 50)
    xy[1:] = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(qlo, qhi + 1, size=(S, n)).astype(np.int32)
    dist = wl.dist_matrix_f32(xy) if dist_mode else None
    return tour, xy, dist, q


@pytest.mark.parametrize("algo", ["plain", "deque", "pipe"])
@pytest.mark.parametrize("beta", [0.0, 0.7, 5.0, 60.0])
def test_soft_c1_vs_oracle(algo, beta):
    """n=50, Q=100, S=1000 Poisson(10) demands (the small Split workload)."""
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    q = wl.split_demands(spec)
    Q = 40  # tighter than the workload's so that overloads pay off at small beta
    orc = oracle.split_soft(tour, Q, beta, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32", algo=algo,
                         overload_penalty=beta)
    torch.cuda.synchronize()
    # beta = 0: the closed tour and its many near-ties; costs are still exact
    check_split(r["cost"], r["pred"], orc, min_checked=0.3 if beta > 0 else 0.0)
    assert abs(float(r["mean"]) - orc["mean"]) <= 1e-5 * orc["mean"]
    assert sdp().status() & (sdp().FLAG_INFEASIBLE | sdp().FLAG_DEVICE_CHECK) == 0


@pytest.mark.parametrize("algo", ["plain", "deque", "pipe"])
@pytest.mark.parametrize("case", [
    # (seed, n, S, Q, qlo, qhi, beta, dist)
    (1, 1, 33, 10, 1, 25, 3.0, False),       # n = 1, demands above Q
    (2, 7, 65, 15, 0, 40, 1.5, True),        # zero demands, dist mode
    (3, 37, 200, 40, 1, 60, 0.25, False),    # cheap overloads: long routes
    (4, 64, 97, 300, 1, 200, 2.0, False),    # uint16 rows (Q >= 255)
    (5, 129, 64, 30, 0, 3, 9.0, False),      # windows longer than 255 customers
    (6, 512, 40, 100, 1, 30, 4.0, False),    # the longest uint8 row the deque stages
    (7, 250, 70, 200, 150, 240, 0.5, False),  # every route overloaded
])
def test_soft_edge_cases(algo, case):
    seed, n, S, Q, qlo, qhi, beta, dm = case
    tour, xy, dist, q = _case(seed, n, S, qlo, qhi, dm)
    kw = {"dist": dist} if dm else {"coords": xy}
    orc = oracle.split_soft(tour, Q, beta, q, want_margin=True, **kw)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), preds="i32", algo=algo, overload_penalty=beta,
                         **{k: _cuda(v) for k, v in kw.items()})
    torch.cuda.synchronize()
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)
    assert abs(float(r["mean"]) - orc["mean"]) <= 1e-5 * abs(orc["mean"])
    assert sdp().status() & sdp().FLAG_INFEASIBLE == 0


@pytest.mark.parametrize("algo", ["deque", "pipe"])
def test_soft_staging_overflow_goes_to_plain(algo):
    """Q <= 254 stages demands as uint8: a row holding a demand of 300 cannot
    be staged and is recomputed by the plain kernel."""
    tour, xy, _, q = _case(11, 40, 70, 1, 30)
    q[5, 7] = 300
    q[64, 0] = 254
    Q, beta = 100, 3.0
    orc = oracle.split_soft(tour, Q, beta, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32", algo=algo,
                         overload_penalty=beta)
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)


@pytest.mark.parametrize("preds", ["u16", "i32", None])
@pytest.mark.parametrize("case", [
    # (seed, n, S, Q, qlo, qhi, beta)
    (21, 50, 300, 40, 1, 20, 5.0),
    (22, 301, 250, 120, 1, 30, 0.7),       # ragged tail, several tiles
    (23, 500, 160, 200, 1, 30, 10.0),      # the benchmark's shape
    (24, 200, 96, 100, 0, 160, 2.0),       # demands above Q (checked step), zeros
    (25, 256, 70, 300, 1, 200, 3.0),       # uint16 rows
    (26, 97, 64, 60, 1, 20, 0.0),          # beta = 0
])
def test_soft_pipe_bit_identical_to_deque(case, preds):
    """The pipelined soft step does the DEQUE soft kernel's FP32 operations:
    where neither recomputes a scenario, costs and predecessors are the same
    bits."""
    seed, n, S, Q, qlo, qhi, beta = case
    tour, xy, _, q = _case(seed, n, S, qlo, qhi)
    args = (_cuda(tour), Q, _cuda(q))
    sdp().status()
    r = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="pipe", overload_penalty=beta)
    d = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="deque", overload_penalty=beta)
    torch.cuda.synchronize()
    assert sdp().status() & (sdp().FLAG_FALLBACK | sdp().FLAG_DEVICE_CHECK | sdp().FLAG_INFEASIBLE) == 0
    assert torch.equal(r["cost"], d["cost"])
    if preds:
        assert torch.equal(r["pred"], d["pred"])
    assert float(r["mean"]) == float(d["mean"])


def test_soft_pipe_prefix_load_past_16_bits():
    """Total demands beyond 2^16: the pipelined kernel's entries keep L(p)
    modulo 2^16, so those scenarios are recomputed by the plain kernel; the
    results stay the oracle's within tolerance."""
    n, S, Q, beta = 900, 64, 400, 2.0
    tour, xy, _, q = _case(31, n, S, 40, 140)
    q[::2] //= 4  # half the scenarios stay below 2^16 in total
    assert (q.sum(1) >= 65536).any() and (q.sum(1) < 65536).any()
    orc = oracle.split_soft(tour, Q, beta, q, coords=xy, want_margin=True)
    sdp().status()
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32", algo="pipe",
                         overload_penalty=beta)
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)


def test_soft_host_demands_chunked():
    """Soft capacity with demands in pinned host memory (copied in 65,536-
    scenario chunks behind the evaluation, the last one ragged): the same
    bits as the call on device demands, whichever kernel AUTO runs."""
    rng = np.random.default_rng(51)
    n, S, Q, beta = 40, 140_003, 60, 3.0
    xy = rng.uniform(0, 100, (n + 1, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 25, size=(S, n)).astype(np.int32)
    q[11, 5] = 90  # above Q: allowed, it pays the penalty
    t, c = _cuda(tour), _cuda(xy)
    ref = sdp().split_eval(t, Q, _cuda(q), coords=c, preds="u16", overload_penalty=beta)
    r = sdp().split_eval(t, Q, torch.from_numpy(q).pin_memory(), coords=c, preds="u16",
                         overload_penalty=beta)
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"]) and torch.equal(r["pred"], ref["pred"])
    assert float(r["mean"]) == float(ref["mean"])
    assert sdp().status() & sdp().FLAG_INFEASIBLE == 0


def test_soft_auto_takes_pipe():
    api = sdp()
    tour, xy, _, q = _case(41, 400, 500, 1, 30)
    args = (_cuda(tour), 150, _cuda(q))
    r = api.split_eval(*args, coords=_cuda(xy), preds="u16", overload_penalty=4.0)
    assert api.last_launch()[0] == 32
    d = api.split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque", overload_penalty=4.0)
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], d["cost"]) and torch.equal(r["pred"], d["pred"])


def test_soft_equals_hard_without_overflow():
    """Q at least the total demand of every scenario: nothing ever leaves the
    window, so the soft DEQUE run is the hard one bit for bit."""
    tour, xy, _, q = _case(12, 60, 300, 1, 9)
    Q = int(q.sum(axis=1).max())
    args = (_cuda(tour), Q, _cuda(q))
    h = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque")
    s = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque", overload_penalty=4.0)
    torch.cuda.synchronize()
    assert torch.equal(h["cost"], s["cost"]) and torch.equal(h["pred"], s["pred"])


def test_soft_rejections():
    api = sdp()
    tour, xy, dist, q = _case(13, 600, 4, 1, 9, dist_mode=True)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    for kw, code in ((dict(algo="stream", overload_penalty=1.0), -5),
                     (dict(algo="deque", overload_penalty=1.0), -5),   # 600 B rows
                     (dict(algo="plain", overload_penalty=-1.0), -1)):
        with pytest.raises(api.SdpError) as e:
            api.split_eval(t, 50, qd, coords=c, **kw)
        assert e.value.code == code
    # AUTO takes the pipelined kernel for rows the deque cannot stage
    r = api.split_eval(t, 50, qd, coords=c, overload_penalty=1.0, preds="i32")
    assert api.last_launch()[0] == 32
    torch.cuda.synchronize()
    orc = oracle.split_soft(tour, 50, 1.0, q, coords=xy, want_margin=True)
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)


def test_soft_full_size_sampled():
    """n=500, Q=200, S=10^6 U{1..30} demands (the Split bench workload) with a
    penalty of 10 per unit of overload, DEQUE with uint16 predecessors;
    sampled scenarios checked one by one against the oracle."""
    spec = wl.SPLIT_C2
    tour, xy, _ = wl.split_tour(spec)
    qd = wl.split_demands_device(spec)
    beta = 10.0
    r = sdp().split_eval(_cuda(tour), spec.Q, qd, coords=_cuda(xy), preds="u16", algo="deque",
                         overload_penalty=beta)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2)
    rows = np.sort(rng.choice(spec.S, 300, replace=False))
    rows = np.concatenate([rows, [0, spec.S - 1]])
    qs = np.concatenate([wl.split_demands(spec, int(s), int(s) + 1) for s in rows])
    orc = oracle.split_soft(tour, spec.Q, beta, qs, coords=xy, want_margin=True)
    check_split(r["cost"], r["pred"], orc, rows=rows, margin=1e-5, min_checked=0.5)
    hard = sdp().split_eval(_cuda(tour), spec.Q, qd, coords=_cuda(xy), algo="deque")
    torch.cuda.synchronize()
    assert bool((r["cost"] <= hard["cost"] * (1 + 1e-6)).all())  # overloads only help
    assert sdp().status() & (sdp().FLAG_INFEASIBLE | sdp().FLAG_FALLBACK) == 0

"""GPU parity of the pipelined Split path (SDP_ALGO_PIPE: producer warps
narrow and permute each tile's demand rows into tour order in an L2-resident
slot ring, 23 DP warps per SM run the deque step, predecessors leave through
a shared-memory transpose) against the FP64 oracle and, bit for bit, against
the PLAIN and DEQUE kernels, through the C ABI."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.golden_io import arr, load
from tests.gpu_util import check_split, preds_to_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_pipe_paper_toy():
    g = load("split_toy.json")
    dist = np.asarray(g["cost_matrix"], np.float32)
    tour = arr(g["tour"], np.int32)
    q = arr(g["demand_by_customer"], np.int32)[None, :]
    r = sdp().split_eval(_cuda(tour), g["Q"], _cuda(q), dist=_cuda(dist), preds="i32",
                         algo="pipe")
    torch.cuda.synchronize()
    assert float(r["cost"][0]) == g["V"][-1]
    assert preds_to_i64(r["pred"])[0].tolist() == g["pred"]


@pytest.mark.parametrize("preds", ["u16", "i32", None])
def test_pipe_c1_full(preds):
    """n=50, S=1000 against the oracle (1000 = 31 tiles + 8 rows; 50 = 3
    blocks of 16 positions + a ragged tail of 2)."""
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    q = wl.split_demands(spec)
    orc = oracle.split(tour, spec.Q, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), spec.Q, _cuda(q), coords=_cuda(xy), preds=preds,
                         algo="pipe")
    torch.cuda.synchronize()
    check_split(r["cost"], r["pred"], orc)
    assert abs(float(r["mean"]) - orc["mean"]) <= 1e-5 * orc["mean"]
    assert sdp().status() & (sdp().FLAG_INFEASIBLE | sdp().FLAG_DEVICE_CHECK) == 0


@pytest.mark.parametrize("case", [
    # (seed, n, S, Q, qlo, qhi, dist)
    (1, 1, 33, 10, 1, 10, False),        # n = 1: tail only
    (2, 3, 70, 10, 1, 12, False),        # some infeasible (demand > Q)
    (3, 7, 65, 15, 0, 9, True),          # zero demands, dist mode
    (4, 37, 200, 40, 1, 45, False),      # infeasible scenarios, odd n
    (5, 64, 97, 255, 1, 60, False),      # uint16 rows (Q >= 255)
    (6, 129, 64, 300, 0, 3, False),      # long windows: > 255 customers per route
    (7, 250, 131, 30000, 1, 500, False),  # uint16, large Q, long routes
    (8, 600, 70, 200, 1, 30, False),     # longer than a tensor-memory row
    (9, 256, 96, 30000, 1, 600, False),  # uint16, loads above 2^16 (wrap)
    (10, 300, 64, 254, 200, 254, False),  # uint8, loads above 2^16 (wrap)
    (11, 1000, 40, 150, 1, 151, False),  # a few demands of Q + 1
    (12, 1024, 33, 32767, 1, 9000, False),  # the largest n and Q
    (13, 999, 45, 600, 1, 700, False),   # uint16 rows, odd n, infeasible rows
])
def test_pipe_edge_cases(case):
    seed, n, S, Q, qlo, qhi, dm = case
    tour, xy, dist, q = _case(seed, n, S, Q, qlo, qhi, dm)
    kw = {"dist": dist} if dm else {"coords": xy}
    orc = oracle.split(tour, Q, q, want_margin=True, **kw)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), preds="i32", algo="pipe",
                         **{k: _cuda(v) for k, v in kw.items()})
    torch.cuda.synchronize()
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)
    if np.isinf(orc["cost"]).any():
        assert np.isinf(float(r["mean"]))
        assert sdp().status() & sdp().FLAG_INFEASIBLE
    else:
        assert abs(float(r["mean"]) - orc["mean"]) <= 1e-5 * abs(orc["mean"])
        assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 31, 33, 64, 100, 170, 171, 250, 340, 341,
                               500, 513, 1000, 1024])
@pytest.mark.parametrize("Q,hi", [(60, 20), (600, 80)])
def test_pipe_bit_identical_to_deque_and_plain(n, Q, hi):
    """Every block / tail split of the row, uint8 and uint16 rows, uint16
    predecessor pairs on odd and even n and int32 predecessors give the bits
    of the other two kernels; S = 257 leaves a ragged last tile.  n = 170 /
    171 (uint16) and 340 / 341 (uint8) are the rows of 85 and 86 words on
    either side of the narrowing's switch from row groups over all its
    threads to one thread per word position."""
    tour, xy, _, q = _case(100 + n, n, 257, Q, 1, hi)
    args = (_cuda(tour), Q, _cuda(q))
    for preds in ("u16", "i32"):
        ref = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="plain")
        dq = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="deque")
        pp = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="pipe")
        torch.cuda.synchronize()
        assert torch.equal(pp["cost"], ref["cost"]) and torch.equal(pp["cost"], dq["cost"])
        assert torch.equal(pp["pred"], ref["pred"]) and torch.equal(pp["pred"], dq["pred"])
        assert float(pp["mean"]) == float(ref["mean"])
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("S", [1, 31, 32, 33, 511, 512, 513, 16 * 32 * 152 + 17])
def test_pipe_scenario_counts(S):
    """Tile and group boundaries of the work queue: one scenario, partial
    tiles, exact groups, and more groups than SMs with a ragged tail."""
    tour, xy, _, q = _case(7 + S, 96, S, 80, 1, 25)
    args = (_cuda(tour), 80, _cuda(q))
    ref = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque")
    pp = sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo="pipe")
    torch.cuda.synchronize()
    assert torch.equal(pp["cost"], ref["cost"])
    assert torch.equal(pp["pred"], ref["pred"])
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("pred_dtype", ["u16", "i32"])
def test_pipe_unaligned_pred_output(pred_dtype):
    """A predecessor array one element off its allocation's alignment takes
    the halfword store path (uint16); results equal the aligned call and the
    element before the array is untouched."""
    api = sdp()
    tour, xy, _, q = _case(5, 64, 300, 50, 1, 15)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    ref = api.split_eval(t, 50, qd, coords=c, preds=pred_dtype, algo="pipe")
    S, n = q.shape
    buf = torch.full((S * n + 1,), -7, dtype=ref["pred"].dtype, device="cuda")
    pred = buf[1:].view(S, n)
    cost = torch.empty(S, dtype=torch.float32, device="cuda")
    a = api._split_struct(t, 50, qd, c, None, cost, pred, api.PRED_DTYPES[pred_dtype],
                          "pipe", None, 0, 0)
    lib = api._load()
    ws = torch.empty(lib.sdp_split_workspace_bytes(ctypes.byref(a)), dtype=torch.uint8,
                     device="cuda")
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    assert lib.sdp_split_eval(ctypes.byref(a), None) == 0
    torch.cuda.synchronize()
    assert torch.equal(cost, ref["cost"])
    assert torch.equal(pred, ref["pred"])
    assert int(buf[0]) == -7


def test_pipe_ring_overflow_fallback():
    """All travel costs zero: every candidate ties and stays in the deque, so
    windows longer than the ring send those scenarios to the plain kernel."""
    n, S, Q = 40, 70, 40
    rng = np.random.default_rng(9)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, 3, size=(S, n)).astype(np.int32)
    xy = np.full((n + 1, 2), 50.0, np.float32)
    orc = oracle.split(tour, Q, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32",
                         algo="pipe")
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    np.testing.assert_array_equal(preds_to_i64(r["pred"]), orc["pred"])
    np.testing.assert_array_equal(r["cost"].cpu().numpy(), 0.0)


def test_pipe_monotone_window_overflow():
    """Customers on a ray from the depot, zero demands: psi rises along the
    tour, nothing pops from the back, and the deque outgrows the 14 entries
    the ring test allows; those scenarios are recomputed and match the
    oracle."""
    n, S, Q = 60, 40, 1000
    xy = np.zeros((n + 1, 2), np.float32)
    xy[0] = (0, 0)
    xy[1:, 0] = np.arange(1, n + 1, dtype=np.float32) ** 1.5
    tour = np.arange(1, n + 1, dtype=np.int32)
    q = np.zeros((S, n), np.int32)
    q[::2, ::7] = 1
    orc = oracle.split(tour, Q, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32",
                         algo="pipe")
    ref = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32",
                           algo="plain")
    torch.cuda.synchronize()
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)
    assert torch.equal(r["cost"], ref["cost"]) and torch.equal(r["pred"], ref["pred"])
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


def test_pipe_rejects_unsupported():
    api = sdp()
    n = 1025
    tour = torch.arange(1, n + 1, dtype=torch.int32, device="cuda")
    xy = torch.zeros((n + 1, 2), dtype=torch.float32, device="cuda")
    q = torch.ones((2, n), dtype=torch.int32, device="cuda")
    with pytest.raises(api.SdpError) as e:
        api.split_eval(tour, 10, q, coords=xy, algo="pipe")
    assert e.value.code == -5
    n = 8
    tour = torch.arange(1, n + 1, dtype=torch.int32, device="cuda")
    xy = torch.zeros((n + 1, 2), dtype=torch.float32, device="cuda")
    buf = torch.ones(2 * n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(api.SdpError) as e:
        api.split_eval(tour, 10, buf[1:].view(2, n), coords=xy, algo="pipe")
    assert e.value.code == -5
    # AUTO falls back to another kernel for the same unaligned demands
    r = api.split_eval(tour, 10, buf[1:].view(2, n), coords=xy, preds="i32")
    ref = api.split_eval(tour, 10, buf[1:].view(2, n).clone(), coords=xy, preds="i32",
                         algo="pipe")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"]) and torch.equal(r["pred"], ref["pred"])


def test_pipe_host_demands_chunked():
    """Pinned host demands through the chunked copy pipeline (three chunks,
    the last ragged) give the bits of the device-demand call."""
    rng = np.random.default_rng(22)
    n, S, Q = 24, 150_001, 60
    xy = rng.uniform(0, 100, (n + 1, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 25, size=(S, n)).astype(np.int32)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    qh = torch.from_numpy(q).pin_memory()
    ref = sdp().split_eval(t, Q, qd, coords=c, preds="u16", algo="deque")
    for _ in range(2):
        r = sdp().split_eval(t, Q, qh, coords=c, preds="u16", algo="pipe")
        torch.cuda.synchronize()
        assert torch.equal(r["cost"], ref["cost"])
        assert torch.equal(r["pred"], ref["pred"])


def test_auto_takes_pipe():
    """AUTO runs the pipelined kernel for an aligned device demand array
    (sdp_last_launch reports its 32 warps per CTA) and gives its bits."""
    api = sdp()
    tour, xy, _, q = _case(3, 200, 1000, 120, 1, 20)
    args = (_cuda(tour), 120, _cuda(q))
    r = api.split_eval(*args, coords=_cuda(xy), preds="u16")
    assert api.last_launch()[0] == 32
    ref = api.split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"]) and torch.equal(r["pred"], ref["pred"])


@pytest.mark.parametrize("S", [1, 31, 33, 100, 4096, 152 * 32 + 1, 152 * 32 * 9 + 77])
def test_pipe_launch_spread_and_slots(S):
    """One tour claims its tiles one at a time: a launch has one CTA per tile
    up to the SM count, and each CTA's ring has twice its share of the tiles
    (2 to 32 slots); every spread gives the DEQUE kernel's bits."""
    api = sdp()
    tour, xy, _, q = _case(40 + S % 97, 137, S, 90, 1, 25)
    args = (_cuda(tour), 90, _cuda(q))
    r = api.split_eval(*args, coords=_cuda(xy), preds="u16", algo="pipe")
    warps, ctas = api.last_launch()
    tiles = (S + 31) // 32
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert warps == 32 and ctas == min(sms, tiles)
    ref = api.split_eval(*args, coords=_cuda(xy), preds="u16", algo="deque")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"]) and torch.equal(r["pred"], ref["pred"])
    assert api.status() & (api.FLAG_DEVICE_CHECK | api.FLAG_FALLBACK) == 0


def test_pipe_c2_full_size_sampled():
    """n=500, S=10^6 generated on the device, in the launch configuration the
    benchmark times (PIPE, uint16 predecessors): all scenarios bit-identical
    to the DEQUE kernel, sampled scenarios checked one by one against the
    oracle."""
    spec = wl.SPLIT_C2
    tour, xy, _ = wl.split_tour(spec)
    qd = wl.split_demands_device(spec)
    t, c = _cuda(tour), _cuda(xy)
    r = sdp().split_eval(t, spec.Q, qd, coords=c, preds="u16", algo="pipe")
    ref = sdp().split_eval(t, spec.Q, qd, coords=c, preds="u16", algo="deque")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"])
    assert torch.equal(r["pred"], ref["pred"])
    assert float(r["mean"]) == float(ref["mean"])
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(spec.S, 800, replace=False))
    rows = np.concatenate([rows, [0, 31, 32, spec.S - 1]])
    qs = np.concatenate([wl.split_demands(spec, int(s), int(s) + 1) for s in rows])
    orc = oracle.split(tour, spec.Q, qs, coords=xy, want_margin=True)
    check_split(r["cost"], r["pred"], orc, rows=rows, margin=1e-5, min_checked=0.7)
    assert sdp().status() & (sdp().FLAG_INFEASIBLE | sdp().FLAG_FALLBACK) == 0

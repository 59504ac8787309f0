"""GPU parity of the streaming Split path (SDP_ALGO_STREAM: producer warps
narrow and permute the demand rows into tour order, DP warps of the same CTA
stream them) against the FP64 oracle and, bit for bit, against the PLAIN and
DEQUE kernels, through the C ABI."""
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


def test_stream_paper_toy():
    g = load("split_toy.json")
    dist = np.asarray(g["cost_matrix"], np.float32)
    tour = arr(g["tour"], np.int32)
    q = arr(g["demand_by_customer"], np.int32)[None, :]
    r = sdp().split_eval(_cuda(tour), g["Q"], _cuda(q), dist=_cuda(dist), preds="i32",
                         algo="stream")
    torch.cuda.synchronize()
    assert float(r["cost"][0]) == g["V"][-1]
    assert preds_to_i64(r["pred"])[0].tolist() == g["pred"]


@pytest.mark.parametrize("preds", ["u16", "i32", None])
def test_stream_c1_full(preds):
    """n=50, S=1000 against the oracle (1000 = 31 tiles + 8 rows; 50 = 3
    blocks of 16 positions + a ragged tail of 2; 50 % 4 = 2: pair stores)."""
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    q = wl.split_demands(spec)
    orc = oracle.split(tour, spec.Q, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), spec.Q, _cuda(q), coords=_cuda(xy), preds=preds,
                         algo="stream")
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
    (12, 2048, 33, 32767, 1, 9000, False),  # the largest n and Q
])
def test_stream_edge_cases(case):
    seed, n, S, Q, qlo, qhi, dm = case
    tour, xy, dist, q = _case(seed, n, S, Q, qlo, qhi, dm)
    kw = {"dist": dist} if dm else {"coords": xy}
    orc = oracle.split(tour, Q, q, want_margin=True, **kw)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), preds="i32", algo="stream",
                         **{k: _cuda(v) for k, v in kw.items()})
    torch.cuda.synchronize()
    check_split(r["cost"], r["pred"], orc, min_checked=0.0)
    if np.isinf(orc["cost"]).any():
        assert np.isinf(float(r["mean"]))
        assert sdp().status() & sdp().FLAG_INFEASIBLE
    else:
        assert abs(float(r["mean"]) - orc["mean"]) <= 1e-5 * abs(orc["mean"])
        sdp().status()


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 31, 33, 64, 100, 250, 500, 513])
@pytest.mark.parametrize("Q,hi", [(60, 20), (600, 80)])
def test_stream_bit_identical_to_deque_and_plain(n, Q, hi):
    """Every block / tail split of the row, uint8 and uint16 rows, and the
    three predecessor store widths (n % 4 == 0: 4 per store; n even: 2; odd:
    1) give the bits of the other two kernels."""
    tour, xy, _, q = _case(100 + n, n, 257, Q, 1, hi)
    args = (_cuda(tour), Q, _cuda(q))
    for preds in ("u16", "i32"):
        ref = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="plain")
        dq = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="deque")
        st = sdp().split_eval(*args, coords=_cuda(xy), preds=preds, algo="stream")
        torch.cuda.synchronize()
        assert torch.equal(st["cost"], ref["cost"]) and torch.equal(st["cost"], dq["cost"])
        assert torch.equal(st["pred"], ref["pred"]) and torch.equal(st["pred"], dq["pred"])
        assert float(st["mean"]) == float(ref["mean"])


@pytest.mark.parametrize("n,Q,hi", [(600, 200, 30), (1000, 150, 20), (2000, 150, 20),
                                    (700, 400, 50)])
def test_long_rows_auto_deque_stream_plain_agree(n, Q, hi):
    """Rows longer than the tensor-memory staging: AUTO (which takes STREAM
    here), DEQUE (shared-memory staging with as many warps as fit) and PLAIN
    give the same bits."""
    tour, xy, _, q = _case(7 * n, n, 100, Q, 1, hi)
    args = (_cuda(tour), Q, _cuda(q))
    outs = {algo: sdp().split_eval(*args, coords=_cuda(xy), preds="u16", algo=algo)
            for algo in ("plain", "deque", "stream", "auto")}
    torch.cuda.synchronize()
    for algo in ("deque", "stream", "auto"):
        assert torch.equal(outs[algo]["cost"], outs["plain"]["cost"]), algo
        assert torch.equal(outs[algo]["pred"], outs["plain"]["pred"]), algo
    assert sdp().status() & sdp().FLAG_DEVICE_CHECK == 0


@pytest.mark.parametrize("pred_dtype", ["u16", "i32"])
def test_stream_unaligned_pred_output(pred_dtype):
    """A predecessor array one element off its allocation's alignment takes
    the scalar store path; results equal the aligned call and the element
    before the array is untouched."""
    api = sdp()
    tour, xy, _, q = _case(5, 64, 300, 50, 1, 15)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    ref = api.split_eval(t, 50, qd, coords=c, preds=pred_dtype, algo="stream")
    S, n = q.shape
    buf = torch.full((S * n + 1,), -7, dtype=ref["pred"].dtype, device="cuda")
    pred = buf[1:].view(S, n)
    cost = torch.empty(S, dtype=torch.float32, device="cuda")
    a = api._split_struct(t, 50, qd, c, None, cost, pred, api.PRED_DTYPES[pred_dtype],
                          "stream", None, 0, 0)
    lib = api._load()
    ws = torch.empty(lib.sdp_split_workspace_bytes(ctypes.byref(a)), dtype=torch.uint8,
                     device="cuda")
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    assert lib.sdp_split_eval(ctypes.byref(a), None) == 0
    torch.cuda.synchronize()
    assert torch.equal(cost, ref["cost"])
    assert torch.equal(pred, ref["pred"])
    assert int(buf[0]) == -7


def test_stream_ring_overflow_fallback():
    """All travel costs zero: every candidate ties and stays in the deque, so
    windows longer than the ring send those scenarios to the plain kernel."""
    n, S, Q = 40, 70, 40
    rng = np.random.default_rng(9)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(0, 3, size=(S, n)).astype(np.int32)
    xy = np.full((n + 1, 2), 50.0, np.float32)
    orc = oracle.split(tour, Q, q, coords=xy, want_margin=True)
    r = sdp().split_eval(_cuda(tour), Q, _cuda(q), coords=_cuda(xy), preds="i32",
                         algo="stream")
    torch.cuda.synchronize()
    assert sdp().status() & sdp().FLAG_FALLBACK
    np.testing.assert_array_equal(preds_to_i64(r["pred"]), orc["pred"])
    np.testing.assert_array_equal(r["cost"].cpu().numpy(), 0.0)


def test_stream_rejects_unsupported():
    api = sdp()
    n = 2049
    tour = torch.arange(1, n + 1, dtype=torch.int32, device="cuda")
    xy = torch.zeros((n + 1, 2), dtype=torch.float32, device="cuda")
    q = torch.ones((2, n), dtype=torch.int32, device="cuda")
    with pytest.raises(api.SdpError) as e:
        api.split_eval(tour, 10, q, coords=xy, algo="stream")
    assert e.value.code == -5
    # demands off a 16-byte boundary
    n = 8
    tour = torch.arange(1, n + 1, dtype=torch.int32, device="cuda")
    xy = torch.zeros((n + 1, 2), dtype=torch.float32, device="cuda")
    buf = torch.ones(2 * n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(api.SdpError) as e:
        api.split_eval(tour, 10, buf[1:].view(2, n), coords=xy, algo="stream")
    assert e.value.code == -5


def test_stream_host_demands_chunked():
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
        r = sdp().split_eval(t, Q, qh, coords=c, preds="u16", algo="stream")
        torch.cuda.synchronize()
        assert torch.equal(r["cost"], ref["cost"])
        assert torch.equal(r["pred"], ref["pred"])


def test_stream_c2_full_size_sampled():
    """n=500, S=10^6 generated on the device, in the launch configuration the
    benchmark times (STREAM, uint16 predecessors): all scenarios bit-identical
    to the DEQUE kernel, sampled scenarios checked one by one against the
    oracle."""
    spec = wl.SPLIT_C2
    tour, xy, _ = wl.split_tour(spec)
    qd = wl.split_demands_device(spec)
    t, c = _cuda(tour), _cuda(xy)
    r = sdp().split_eval(t, spec.Q, qd, coords=c, preds="u16", algo="stream")
    ref = sdp().split_eval(t, spec.Q, qd, coords=c, preds="u16", algo="deque")
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"])
    assert torch.equal(r["pred"], ref["pred"])
    assert float(r["mean"]) == float(ref["mean"])
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(spec.S, 800, replace=False))
    rows = np.concatenate([rows, [0, 31, 32, spec.S - 1]])
    qs = np.concatenate([wl.split_demands(spec, int(s), int(s) + 1) for s in rows])
    orc = oracle.split(tour, spec.Q, qs, coords=xy, want_margin=True)
    check_split(r["cost"], r["pred"], orc, rows=rows, margin=1e-5, min_checked=0.7)
    assert sdp().status() & (sdp().FLAG_INFEASIBLE | sdp().FLAG_FALLBACK) == 0

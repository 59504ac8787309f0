"""sdp_split_eval_noalloc: the Split entry point for callers that cannot give
the library any device memory besides their inputs and outputs (it uses a
fixed scratch array inside the library instead of a caller workspace).

Checked through the C ABI against the ordinary entry point (sdp_split_eval)
on the same inputs, on two calls in a row with different shapes, and the
rejection of calls whose scratch would not fit.  This file is collected last
so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.gpu_util import check_split, preds_to_i64

torch = pytest.importorskip("torch")

SDP_ERR_UNSUPPORTED = -5


def _lib():
    from paper_2602_05179_gb300 import api
    lib = ctypes.CDLL(api.lib_path())
    lib.sdp_split_eval_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.sdp_split_eval_noalloc.restype = ctypes.c_int
    lib.sdp_last_error.restype = ctypes.c_char_p
    return api, lib


def _noalloc(tour, Q, demands, coords=None, dist=None, preds=True):
    """Outputs allocated by the caller; no workspace passed."""
    api, lib = _lib()
    S, n = demands.shape
    cost = torch.empty(S, dtype=torch.float32, device="cuda")
    pred = torch.empty((S, n), dtype=torch.int32, device="cuda") if preds else None
    mean = torch.empty((), dtype=torch.float64, device="cuda")
    a = api._split_struct(tour, Q, demands, coords, dist, cost, pred,
                          api.PRED_DTYPES["i32"] if preds else 0, "auto", mean, 0, 0)
    a.workspace, a.workspace_bytes = None, 0
    rc = lib.sdp_split_eval_noalloc(ctypes.byref(a),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, (rc, lib.sdp_last_error())
    return cost, pred, mean


def test_noalloc_rejects_oversize_without_touching_the_device():
    from paper_2602_05179_gb300 import api
    import os
    if not os.path.exists(api.lib_path()):
        pytest.skip("libsdp.so is not built")
    try:
        api, lib = _lib()
    except OSError as e:  # a library that does not load here (no CUDA runtime)
        pytest.skip(f"libsdp.so does not load: {e}")
    a = api.SplitArgs()
    a.n, a.Q, a.S, a.algo = 500, 200, 100_000_000, 0
    rc = lib.sdp_split_eval_noalloc(ctypes.byref(a), None)
    assert rc == SDP_ERR_UNSUPPORTED
    assert b"no-allocation scratch" in lib.sdp_last_error()


@pytest.mark.gpu
def test_noalloc_matches_eval_two_calls_in_a_row():
    api, _ = _lib()
    # call 1: the n=50, S=1000 workload
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    q = wl.split_demands(spec)
    t, c, qd = (torch.from_numpy(x).cuda() for x in (tour, xy, q))
    ref = api.split_eval(t, spec.Q, qd, coords=c, preds="i32")
    cost, pred, mean = _noalloc(t, spec.Q, qd, coords=c)
    torch.cuda.synchronize()
    orc = oracle.split(tour, spec.Q, q, coords=xy, want_margin=True)
    check_split(cost, pred, orc)
    np.testing.assert_allclose(cost.cpu().numpy(), ref["cost"].cpu().numpy(), rtol=1e-5)
    assert torch.equal(pred, ref["pred"])
    assert abs(float(mean) - float(ref["mean"])) <= 1e-5 * abs(float(ref["mean"]))

    # call 2, right after: another shape, with infeasible scenarios, so that
    # anything left over from call 1 in the shared scratch would show
    rng = np.random.default_rng(5)
    n2, S2, Q2 = 37, 203, 40
    xy2 = np.concatenate([[[50, 50]], rng.uniform(0, 100, (n2, 2))]).astype(np.float32)
    tour2 = (rng.permutation(n2) + 1).astype(np.int32)
    q2 = rng.integers(1, 45, size=(S2, n2)).astype(np.int32)
    t2, c2, qd2 = (torch.from_numpy(x).cuda() for x in (tour2, xy2, q2))
    ref2 = api.split_eval(t2, Q2, qd2, coords=c2, preds="i32")
    cost2, pred2, mean2 = _noalloc(t2, Q2, qd2, coords=c2)
    torch.cuda.synchronize()
    orc2 = oracle.split(tour2, Q2, q2, coords=xy2, want_margin=True)
    check_split(cost2, pred2, orc2, min_checked=0.0)
    a, b = cost2.cpu().numpy(), ref2["cost"].cpu().numpy()
    assert np.array_equal(np.isinf(a), np.isinf(b))
    f = np.isfinite(b)
    np.testing.assert_allclose(a[f], b[f], rtol=1e-5)
    assert np.array_equal(preds_to_i64(pred2), preds_to_i64(ref2["pred"]))
    assert np.isinf(float(mean2)) == np.isinf(float(ref2["mean"]))
    api.status()


@pytest.mark.gpu
def test_noalloc_rejects_host_demands_beyond_the_scratch():
    """Page-locked host demands need two staging buffers of min(S, 65536) * n
    int32 each: at n = 64 and S = 65536 they alone exceed the scratch, so the
    call is rejected before anything is launched."""
    api, lib = _lib()
    n, S = 64, 65536
    rng = np.random.default_rng(9)
    xy = np.concatenate([[[50, 50]], rng.uniform(0, 100, (n, 2))]).astype(np.float32)
    tour = torch.from_numpy((rng.permutation(n) + 1).astype(np.int32)).cuda()
    q = torch.ones((S, n), dtype=torch.int32).pin_memory()
    cost = torch.empty(S, dtype=torch.float32, device="cuda")
    a = api._split_struct(tour, 100, q, torch.from_numpy(xy).cuda(), None, cost, None, 0,
                          "auto", None, 0, 0)
    rc = lib.sdp_split_eval_noalloc(ctypes.byref(a), None)
    assert rc == SDP_ERR_UNSUPPORTED
    assert b"no-allocation scratch" in lib.sdp_last_error()

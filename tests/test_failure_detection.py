"""Failure detection without a GPU fault: injected host-side errors (the
allocator, the launch of an operator call, an out-of-memory result), the
adaptive batching of Algorithm "GPU-Based DP with Adaptive Batching" (halve
the batch on out-of-memory and retry), and the streaming kernels' bounded
device waits made to run out by a producer that publishes nothing.  No test
faults, traps or hangs a GPU: every injected failure is an error code
returned before a launch, or a wait that gives up after a short limit."""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _lib_or_skip():
    api = sdp()
    if not os.path.exists(api.lib_path()):
        pytest.skip("libsdp.so is not built")
    try:
        return api._load()
    except OSError as e:
        pytest.skip(f"libsdp.so does not load: {e}")


# ------------------------------------------------------------------ host side
def test_adaptive_batches_halves_on_out_of_memory():
    api = sdp()
    calls = []

    def run(s0, s1):
        calls.append((s0, s1))
        if s1 - s0 > 100:
            raise api.SdpError(api.ERR_OOM, "fake out-of-memory")
        return np.arange(s0, s1)

    parts, sizes = api.adaptive_batches(run, 1000, batch=1000)
    assert sizes == [1000, 500, 250, 125, 62]
    # the slices cover [0, 1000) in order, each retried slice starting where
    # the failed one did
    assert [p[0] for p in parts][0] == 0 and parts[-1][1] == 1000
    assert all(a[1] == b[0] for a, b in zip(parts[:-1], parts[1:]))
    np.testing.assert_array_equal(np.concatenate([p[2] for p in parts]), np.arange(1000))
    assert calls[:4] == [(0, 1000), (0, 500), (0, 250), (0, 125)]


def test_adaptive_batches_other_errors_and_floor():
    api = sdp()

    def bad(s0, s1):
        raise api.SdpError(api.ERR_CUDA, "not an allocation failure")
    with pytest.raises(api.SdpError) as e:
        api.adaptive_batches(bad, 64, batch=64)
    assert e.value.code == api.ERR_CUDA

    def never(s0, s1):
        raise api.SdpError(api.ERR_OOM, "fake")
    with pytest.raises(api.SdpError):  # stops at min_batch instead of looping
        api.adaptive_batches(never, 64, batch=64, min_batch=8)
    parts, sizes = api.adaptive_batches(lambda a, b: b - a, 0, batch=16)
    assert parts == []


def test_fault_spec_is_checked_on_the_host():
    lib = _lib_or_skip()
    lib.sdp_set_fault_inject.argtypes = [ctypes.c_char_p]
    lib.sdp_set_fault_inject.restype = ctypes.c_int
    lib.sdp_last_error.restype = ctypes.c_char_p
    for bad in (b"bogus", b"alloc:x", b"stall", b"oom:-1"):
        assert lib.sdp_set_fault_inject(bad) == -1, bad
        assert b"bad fault spec" in lib.sdp_last_error()
    for good in (b"alloc", b"launch:2,oom:1", b"stall:1000", b"none"):
        assert lib.sdp_set_fault_inject(good) == 0, good
    assert lib.sdp_set_fault_inject(None) == 0


# ------------------------------------------------------------------ on a GPU
def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture
def clean_faults():
    yield
    sdp().set_fault_inject(None)


@pytest.mark.gpu
def test_injected_oom_halves_the_reinsertion_batch(clean_faults):
    """Two injected out-of-memory results: the batched evaluation halves its
    batch twice and then matches the single call bit for bit."""
    api = sdp()
    rng = np.random.default_rng(3)
    S, T, U = 1000, 30, 80
    cons = _cuda(rng.poisson(8.0, size=(S, T)).astype(np.int32))
    fixed = _cuda(rng.uniform(5, 50, T).astype(np.float32))
    ref = api.reinsert_eval(T, U, 40, 1.0, 20.0, 0.0, fixed, cons)
    api.set_fault_inject("oom:2")
    r = api.reinsert_eval_batched(T, U, 40, 1.0, 20.0, 0.0, fixed, cons, batch=S)
    torch.cuda.synchronize()
    assert r["batches"] == [S, S // 2, S // 4]
    assert torch.equal(r["value"], ref["value"]) and torch.equal(r["policy"], ref["policy"])
    assert abs(float(r["mean"]) - float(ref["mean"])) <= 1e-9 * abs(float(ref["mean"]))


@pytest.mark.gpu
def test_injected_launch_failure_and_recovery(clean_faults):
    api = sdp()
    rng = np.random.default_rng(4)
    n, S, Q = 40, 300, 60
    xy = np.vstack([[50.0, 50.0], rng.uniform(0, 100, (n, 2))]).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 20, size=(S, n)).astype(np.int32)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    ref = api.split_eval(t, Q, qd, coords=c)
    api.set_fault_inject("launch")
    with pytest.raises(api.SdpError) as e:
        api.split_eval(t, Q, qd, coords=c)
    assert e.value.code == api.ERR_CUDA
    r = api.split_eval(t, Q, qd, coords=c)  # one-shot: the next call runs
    torch.cuda.synchronize()
    assert torch.equal(r["cost"], ref["cost"])


@pytest.mark.gpu
def test_injected_allocation_failure_of_a_plan(clean_faults):
    api = sdp()
    rng = np.random.default_rng(5)
    nb = np.array([30, 45], np.int32)
    S, Q = 64, 60
    tours = [(rng.permutation(k) + 1).astype(np.int32) for k in nb]
    coords = [np.vstack([[50.0, 50.0], rng.uniform(0, 100, (k, 2))]).astype(np.float32)
              for k in nb]
    dem = np.concatenate([rng.integers(1, 20, size=(S, k)).astype(np.int32).ravel() for k in nb])
    args = (nb, _cuda(np.concatenate(tours)), _cuda(np.concatenate(coords)), _cuda(dem), Q, S)
    api.set_fault_inject("alloc")
    with pytest.raises(api.SdpError) as e:
        api.SplitPlan(*args)
    assert e.value.code == api.ERR_OOM
    plan = api.SplitPlan(*args)
    costs, _ = plan.run()
    torch.cuda.synchronize()
    assert torch.isfinite(costs).all()
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("algo", ["stream", "pipe"])
def test_streaming_wait_runs_out_and_reports(clean_faults, algo):
    """A streaming or pipelined launch whose producers publish no tile: the
    DP warps give up after 1 ms, the call returns, the status reports a
    device check, and the next launch is correct."""
    api = sdp()
    rng = np.random.default_rng(6)
    n, S, Q = 600, 4096, 150
    xy = np.vstack([[50.0, 50.0], rng.uniform(0, 100, (n, 2))]).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 20, size=(S, n)).astype(np.int32)
    t, c, qd = _cuda(tour), _cuda(xy), _cuda(q)
    ref = api.split_eval(t, Q, qd, coords=c, algo="deque")
    torch.cuda.synchronize()
    api.status()
    api.set_fault_inject("stall:1000000")
    api.split_eval(t, Q, qd, coords=c, algo=algo)
    with pytest.raises(api.SdpError) as e:
        api.status()  # synchronises: the launch has returned
    assert e.value.code == api.ERR_DEVICE_CHECK
    r = api.split_eval(t, Q, qd, coords=c, algo=algo)
    torch.cuda.synchronize()
    assert api.status() & api.FLAG_DEVICE_CHECK == 0
    assert torch.equal(r["cost"], ref["cost"])

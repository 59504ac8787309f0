"""The C ABI's argument checks, on the host (no GPU needed): every entry
point rejects what include/sdp.h says it rejects, with the status code it
names (SDP_ERR_INVALID_ARG = -1 for a bad argument, SDP_ERR_UNSUPPORTED = -5
for a valid one the library does not take), before any device work.
Ordinary host buffers stand in for the arrays: they are neither device
memory nor page-locked host memory, so the pointer checks refuse them."""
import ctypes
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INVALID, UNSUPPORTED = -1, -5
AUTO, PLAIN, DEQUE, STREAM, PIPE = 0, 1, 2, 3, 4
HARD, SOFT = 0, 1
U16, I32 = 1, 2


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05179_gb300 import api
    try:
        lib = ctypes.CDLL(api.lib_path())
    except OSError as e:  # a library that does not load here (no CUDA runtime)
        pytest.skip(f"libsdp.so does not load: {e}")
    P = ctypes.c_void_p
    lib.sdp_last_error.restype = ctypes.c_char_p
    lib.sdp_split_eval.argtypes = [P, P]
    lib.sdp_split_fleet_eval.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.sdp_split_backward.argtypes = [P, P, P, P, P, P]
    lib.sdp_reinsert_eval.argtypes = [P, P]
    return lib


BUF = (ctypes.c_int64 * 4096)()
HOST = ctypes.addressof(BUF)


def _split(**kw):
    from paper_2602_05179_gb300 import api
    a = api.SplitArgs()
    a.n, a.Q, a.S, a.algo = 10, 30, 4, AUTO
    a.tour = a.coords = a.demands = a.cost_out = HOST
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def _expect(lib, rc, code, words):
    assert rc == code, (rc, lib.sdp_last_error())
    msg = lib.sdp_last_error().decode()
    assert words in msg, msg


@pytest.mark.parametrize("kw,code,words", [
    (dict(n=-1), INVALID, "n = -1"),
    (dict(Q=0), INVALID, "Q = 0"),
    (dict(S=-1), INVALID, "S = -1"),
    (dict(S=1 << 32), UNSUPPORTED, "S above"),
    (dict(algo=9), INVALID, "unknown algo"),
    (dict(algo=PIPE, n=1025), UNSUPPORTED, "PIPE needs"),
    (dict(algo=PIPE, Q=40000), UNSUPPORTED, "PIPE needs"),
    (dict(algo=PIPE, demands=HOST + 4), UNSUPPORTED, "16-byte aligned"),
    (dict(algo=DEQUE, Q=40000), UNSUPPORTED, "DEQUE needs"),
    (dict(algo=STREAM, n=3000), UNSUPPORTED, "STREAM needs"),
    (dict(algo=STREAM, demands=HOST + 4), UNSUPPORTED, "16-byte aligned"),
    (dict(capacity_mode=3), INVALID, "unknown capacity_mode"),
    (dict(capacity_mode=SOFT, overload_penalty=-1.0), INVALID, "overload_penalty"),
    (dict(capacity_mode=SOFT, overload_penalty=math.nan), INVALID, "overload_penalty"),
    (dict(capacity_mode=SOFT, overload_penalty=math.inf), INVALID, "overload_penalty"),
    (dict(capacity_mode=SOFT, overload_penalty=1.0, algo=STREAM), UNSUPPORTED,
     "soft capacity runs on"),
    ({}, INVALID, "cost_out must be a device pointer"),
    (dict(S=0, pred_out=HOST, pred_dtype=7), INVALID, "pred_dtype"),
    (dict(S=0, n=65535, pred_out=HOST, pred_dtype=U16), UNSUPPORTED, "uint16 predecessors"),
    (dict(S=0, warps_per_cta=9), INVALID, "warps_per_cta"),
    (dict(S=0, ring=12), INVALID, "ring must be"),
])
def test_split_eval_rejections(lib, kw, code, words):
    _expect(lib, lib.sdp_split_eval(ctypes.byref(_split(**kw)), None), code, words)


def test_split_eval_null_args(lib):
    _expect(lib, lib.sdp_split_eval(None, None), INVALID, "args is NULL")


@pytest.mark.parametrize("kw,K,code,words", [
    (dict(S=0), 0, UNSUPPORTED, "max_routes = 0"),
    (dict(S=0), 65, UNSUPPORTED, "max_routes = 65"),
    (dict(S=0, n=20000), 4, UNSUPPORTED, "n <= 16384"),
    (dict(S=0, capacity_mode=SOFT, overload_penalty=1.0), 4, UNSUPPORTED, "hard capacity"),
    (dict(S=0, pred_out=HOST, pred_dtype=I32), 4, INVALID, "returns routes"),
    (dict(S=0, algo=DEQUE), 4, UNSUPPORTED, "AUTO or PLAIN"),
    ({}, 4, INVALID, "cost_out must be a device pointer"),
])
def test_split_fleet_rejections(lib, kw, K, code, words):
    rc = lib.sdp_split_fleet_eval(ctypes.byref(_split(**kw)), K, None, None, None)
    _expect(lib, rc, code, words)


def test_split_backward_rejections(lib):
    a = _split(S=0)
    _expect(lib, lib.sdp_split_backward(ctypes.byref(a), None, HOST, HOST, None, None),
            UNSUPPORTED, "with respect to dist")
    a = _split(S=0, coords=None, dist=HOST, capacity_mode=SOFT, overload_penalty=1.0)
    _expect(lib, lib.sdp_split_backward(ctypes.byref(a), None, HOST, HOST, None, None),
            UNSUPPORTED, "hard capacity only")
    a = _split(S=0, coords=None, dist=HOST)
    _expect(lib, lib.sdp_split_backward(ctypes.byref(a), None, HOST, HOST, None, None),
            INVALID, "grad_mean must be a device pointer")


def _reinsert(**kw):
    from paper_2602_05179_gb300 import api
    a = api.ReinsertArgs()
    a.T, a.U, a.I0, a.S, a.algo = 60, 200, 100, 4, 0
    a.h, a.p = 1.0, 20.0
    a.fixed = a.consumption = a.value_out = HOST
    for k, v in kw.items():
        setattr(a, k, v)
    return a


@pytest.mark.parametrize("kw,code,words", [
    (dict(T=0), INVALID, "T = 0"),
    (dict(T=4097), INVALID, "T = 4097"),
    (dict(U=-1, I0=0), INVALID, "U = -1"),
    (dict(U=1024), INVALID, "U = 1024"),
    (dict(I0=201), INVALID, "I0 = 201"),
    (dict(S=-1), INVALID, "S < 0"),
    (dict(algo=5), INVALID, "unknown reinsertion algo"),
    (dict(n_routes=65), INVALID, "n_routes = 65"),
    (dict(n_routes=2, U=300, I0=0), UNSUPPORTED, "U <= 255"),
    (dict(n_routes=2, end_cost_table=HOST), UNSUPPORTED, "linear end costs"),
    (dict(T=4096, U=1023, I0=0), UNSUPPORTED, "decision words"),
    ({}, INVALID, "fixed must be a device pointer"),
])
def test_reinsert_eval_rejections(lib, kw, code, words):
    _expect(lib, lib.sdp_reinsert_eval(ctypes.byref(_reinsert(**kw)), None), code, words)


def test_reinsert_eval_null_args(lib):
    _expect(lib, lib.sdp_reinsert_eval(None, None), INVALID, "args is NULL")


def _desc(**kw):
    from paper_2602_05179_gb300 import api
    d = api.BatchDesc()
    d.B, d.Q, d.S = 2, 30, 4
    d.n_host = d.tour_off_host = d.coord_off_host = d.dem_off_host = HOST
    d.tours = d.coords = d.demands = d.costs_out = HOST
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,code,words", [
    (dict(B=0), INVALID, "B < 1"),
    (dict(Q=0), UNSUPPORTED, "1 <= Q <= 32767"),
    (dict(Q=40000), UNSUPPORTED, "1 <= Q <= 32767"),
    (dict(S=0), INVALID, "S < 1"),
    (dict(B=1 << 30, S=1 << 62), UNSUPPORTED, "B*S too large"),
    (dict(dem_off_host=None), INVALID, "host offset arrays"),
    (dict(costs_out=None), INVALID, "costs_out must be set"),
])
def test_plan_create_rejections(lib, kw, code, words):
    lib.sdp_split_plan_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p(12345)
    _expect(lib, lib.sdp_split_plan_create(ctypes.byref(_desc(**kw)), ctypes.byref(h)),
            code, words)
    assert not h.value  # no plan handed out


def test_plan_calls_on_a_null_plan(lib):
    P = ctypes.c_void_p
    lib.sdp_split_plan_create.argtypes = [P, P]
    _expect(lib, lib.sdp_split_plan_create(None, None), INVALID, "NULL")
    for name, args in (("sdp_plan_run", (None, None)),
                       ("sdp_plan_info", (None, None, None, None, None)),
                       ("sdp_plan_configure", (None, -2, 16, 1)),
                       ("sdp_plan_kernel_ms", (None, None)),
                       ("sdp_plan_scenarios_per_lane", (None, None)),
                       ("sdp_plan_count_arcs", (None, None, None)),
                       ("sdp_plan_autotune", (None, None, None))):
        f = getattr(lib, name)
        f.argtypes = [P if a is None else ctypes.c_int32 for a in args]
        assert f(*args) == INVALID, name
    lib.sdp_plan_destroy.argtypes = [P]
    lib.sdp_plan_destroy(None)  # a no-op


def test_count_arcs_and_profile_hook_rejections(lib):
    P = ctypes.c_void_p
    lib.sdp_split_count_arcs.argtypes = [P, P, P, P]
    _expect(lib, lib.sdp_split_count_arcs(None, None, None, None), INVALID, "args is NULL")
    a = _split(S=0, n=5)
    _expect(lib, lib.sdp_split_count_arcs(ctypes.byref(a), HOST, None, None), INVALID,
            "arcs_out must be a device pointer")
    _expect(lib, lib.sdp_split_count_arcs(ctypes.byref(a), None, HOST, None), INVALID,
            "total_out must be a device pointer")
    lib.sdp_set_profile_events.argtypes = [P, P]
    _expect(lib, lib.sdp_set_profile_events(HOST, None), INVALID, "both events or neither")
    _expect(lib, lib.sdp_set_profile_events(None, HOST), INVALID, "both events or neither")
    assert lib.sdp_set_profile_events(None, None) == 0

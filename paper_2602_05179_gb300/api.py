"""Python binding of libsdp (include/sdp.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
checks tensor placement and dtypes, allocates outputs and workspaces through
PyTorch's caching allocator, and passes raw device pointers plus the current
CUDA stream across the C ABI.  There is no CPU path: without the library or a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libsdp.so")
_lock = threading.Lock()
_lib = None

SDP_OK = 0
SDP_WARN_INFEASIBLE = 1
FLAG_INFEASIBLE, FLAG_NEG_INPUT, FLAG_DEVICE_CHECK, FLAG_FALLBACK = 1, 2, 4, 8
ALGOS = {"auto": 0, "plain": 1, "deque": 2, "stream": 3, "pipe": 4}
PRED_DTYPES = {"u16": 1, "i32": 2}

P = ctypes.c_void_p


class SplitArgs(ctypes.Structure):
    """Mirror of sdp_split_args (the Split of Eq. eqdpA); the library checks
    its size against this layout when it loads."""
    _fields_ = [("n", ctypes.c_int32), ("Q", ctypes.c_int32), ("S", ctypes.c_int64),
                ("tour", P), ("coords", P), ("dist", P), ("demands", P),
                ("cost_out", P), ("pred_out", P), ("pred_dtype", ctypes.c_int32),
                ("algo", ctypes.c_int32), ("mean_out", P), ("workspace", P),
                ("workspace_bytes", ctypes.c_size_t), ("warps_per_cta", ctypes.c_int32),
                ("ring", ctypes.c_int32), ("capacity_mode", ctypes.c_int32),
                ("overload_penalty", ctypes.c_float)]


class ReinsertArgs(ctypes.Structure):
    """Mirror of sdp_reinsert_args (the reinsertion DP of Eq. eqdp2 /
    Algorithm SolveBatchDP); size-checked like SplitArgs."""
    _fields_ = [("T", ctypes.c_int32), ("U", ctypes.c_int32), ("I0", ctypes.c_int32),
                ("algo", ctypes.c_int32), ("h", ctypes.c_float), ("p", ctypes.c_float),
                ("unit_cost", ctypes.c_float), ("S", ctypes.c_int64), ("fixed", P),
                ("end_cost_table", P), ("consumption", P), ("value_out", P),
                ("policy_out", P), ("value0_out", P), ("mean_out", P), ("workspace", P),
                ("workspace_bytes", ctypes.c_size_t), ("n_routes", ctypes.c_int32),
                ("route_cost", P), ("route_cap", P)]


class BatchDesc(ctypes.Structure):
    """Mirror of sdp_split_batch_desc (a batched Split plan's tours, offsets
    and outputs)."""
    _fields_ = [("B", ctypes.c_int32), ("Q", ctypes.c_int32), ("S", ctypes.c_int64),
                ("n_host", P), ("tour_off_host", P), ("tours", P), ("coord_off_host", P),
                ("coords", P), ("dem_off_host", P), ("demands", P), ("costs_out", P),
                ("means_out", P)]


class SaaSearchDesc(ctypes.Structure):
    """Mirror of sdp_saa_search_desc (the SAA candidate search's instance,
    neighbourhood size, move kinds and seed)."""
    _fields_ = [("n", ctypes.c_int32), ("coords", P), ("Q", ctypes.c_int32),
                ("S", ctypes.c_int64), ("demands", P), ("B", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("moves", ctypes.c_int32), ("tour0", P)]


class SdpError(RuntimeError):
    """A negative status from the library: .code is the SDP_ERR_* value, the
    message is sdp_last_error() of the failing call."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"libsdp error {code}: {msg}")
        self.code = code


def lib_path() -> str:
    """Path of the in-tree libsdp.so this module loads."""
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: run __graft_entry__.build() "
                               "(python -m paper_2602_05179_gb300.build)")
        lib = ctypes.CDLL(_LIB_PATH)
        i32, i64, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "sdp_version": ([], i32),
            "sdp_last_error": ([], ctypes.c_char_p),
            "sdp_device_status": ([i32, P], i32),
            "sdp_split_args_size": ([], sz),
            "sdp_reinsert_args_size": ([], sz),
            "sdp_split_workspace_bytes": ([P], sz),
            "sdp_split_eval": ([P, P], i32),
            "sdp_split_count_arcs": ([P, P, P, P], i32),
            "sdp_split_fleet_workspace_bytes": ([P, i32, i32], sz),
            "sdp_split_fleet_eval": ([P, i32, P, P, P], i32),
            "sdp_split_backward_workspace_bytes": ([P], sz),
            "sdp_split_backward": ([P, P, P, P, P, P], i32),
            "sdp_reinsert_workspace_bytes": ([P], sz),
            "sdp_reinsert_eval": ([P, P], i32),
            "sdp_set_profile_events": ([P, P], i32),
            "sdp_last_launch": ([P, P], i32),
            "sdp_set_fault_inject": ([ctypes.c_char_p], i32),
            "sdp_split_plan_create": ([P, P], i32),
            "sdp_plan_autotune": ([P, P, ctypes.c_char_p], i32),
            "sdp_plan_run": ([P, P], i32),
            "sdp_plan_kernel_ms": ([P, P], i32),
            "sdp_plan_info": ([P, P, P, P, P], i32),
            "sdp_plan_count_arcs": ([P, P, P], i32),
            "sdp_plan_configure": ([P, i32, i32, i32], i32),
            "sdp_plan_scenarios_per_lane": ([P, P], i32),
            "sdp_saa_search_count_arcs": ([P, P, P], i32),
            "sdp_plan_destroy": ([P], None),
            "sdp_saa_search_create": ([P, P], i32),
            "sdp_saa_search_run": ([P, i32, P, P, P], i32),
            "sdp_saa_search_state": ([P, P, P, P], i32),
            "sdp_saa_search_autotune": ([P, P, ctypes.c_char_p], i32),
            "sdp_saa_search_plan_info": ([P, P, P, P, P], i32),
            "sdp_saa_search_destroy": ([P], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        if lib.sdp_split_args_size() != ctypes.sizeof(SplitArgs):
            raise RuntimeError("sdp_split_args layout mismatch")
        if lib.sdp_reinsert_args_size() != ctypes.sizeof(ReinsertArgs):
            raise RuntimeError("sdp_reinsert_args layout mismatch")
        _lib = lib
        return lib


def _check(rc: int):
    if rc < 0:
        msg = _load().sdp_last_error()
        raise SdpError(rc, msg.decode() if msg else "")
    return rc


def _dev_ptr(t, name, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _demands_ptr(t):
    """demands: a CUDA tensor, or a page-locked (pinned) CPU tensor that the
    kernels read over the host link without a staging copy."""
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError("host demands must be in pinned memory (tensor.pin_memory())")
        if t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError("demands must be contiguous int32")
        return t.data_ptr()
    return _dev_ptr(t, "demands", torch.int32)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def set_profile_events(start, stop):
    """Record torch.cuda.Event start/stop around the dominant kernel of this
    thread's next operator call (None, None disables)."""
    if start is not None and (start.cuda_event == 0 or stop.cuda_event == 0):
        # torch creates the CUDA event on its first record()
        start.record()
        stop.record()
    sp = None if start is None else start.cuda_event
    ep = None if stop is None else stop.cuda_event
    _check(_load().sdp_set_profile_events(sp, ep))


def last_launch():
    """(warps per CTA, CTAs) of the DP kernel of this thread's last Split
    evaluation or adjoint call; (0, 0) for the streaming path, (32, CTAs) for
    the pipelined one (23 DP, 1 issuing and 8 narrowing warps)."""
    w, c = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_load().sdp_last_launch(ctypes.byref(w), ctypes.byref(c)))
    return int(w.value), int(c.value)


ERR_CUDA, ERR_OOM, ERR_DEVICE_CHECK = -2, -3, -6


def set_fault_inject(spec):
    """One-shot host-side faults, for failure-detection tests (None clears):
    "alloc[:N]" the next N plan / search allocations fail (SDP_ERR_OOM);
    "launch[:N]" the next N operator calls fail before launching anything
    (SDP_ERR_CUDA); "oom[:N]" the same with SDP_ERR_OOM; "stall:NS" the next
    streaming Split launch publishes no tile, so its DP warps' bounded waits
    give up after NS nanoseconds and raise FLAG_DEVICE_CHECK; comma-separated
    to combine.  SDP_FAULT_INJECT in the environment sets the same at the
    library's first check."""
    _check(_load().sdp_set_fault_inject(None if spec is None else spec.encode()))


def adaptive_batches(run, S, batch=None, *, bytes_per_scenario=0, device=None, min_batch=1):
    """Evaluate scenarios [0, S) in consecutive slices, as Algorithm "GPU-Based
    DP with Adaptive Batching" of the paper does: the batch size comes from the
    free device memory (bytes_per_scenario each, 80% of what is free) unless
    given; a slice whose evaluation runs out of memory (SdpError with
    ERR_OOM, or torch's OutOfMemoryError) is retried with half the batch, down
    to min_batch; unused cached device memory is released after each slice
    (the algorithm's ClearCache).  run(s0, s1) evaluates scenarios s0..s1-1.
    Returns ([(s0, s1, result), ...] in order, [batch sizes used])."""
    def clear():
        if torch.cuda.is_available():
            torch.cuda.empty_cache()
    if batch is None:
        batch = S
        if bytes_per_scenario > 0 and torch.cuda.is_available():
            free = torch.cuda.mem_get_info(device)[0]
            batch = int(0.8 * free) // int(bytes_per_scenario)
    batch = max(min_batch, min(int(batch), max(S, 1)))
    out, sizes = [], [batch]
    s0 = 0
    while s0 < S:
        s1 = min(S, s0 + batch)
        try:
            r = run(s0, s1)
        except (SdpError, torch.cuda.OutOfMemoryError) as e:
            if isinstance(e, SdpError) and e.code != ERR_OOM:
                raise
            if batch <= min_batch:
                raise
            batch = max(min_batch, batch // 2)
            sizes.append(batch)
            clear()
            continue
        out.append((s0, s1, r))
        s0 = s1
        clear()
    return out, sizes


def reinsert_eval_batched(T, U, I0, h, p, unit_cost, fixed, consumption, *, batch=None,
                          min_batch=32, **kw):
    """reinsert_eval (Algorithm SolveBatchDP) over consumption [S, T] in
    adaptive batches (adaptive_batches: the halving on out-of-memory of
    Algorithm gpu-dp): value [S], policy [S, T] (if asked), FP64 mean over
    all S, and the batch sizes used."""
    S = int(consumption.shape[0])
    per = 4 * T + 4 + T + 4 * (U + 1)  # inputs and outputs of one scenario, roughly
    parts, sizes = adaptive_batches(
        lambda s0, s1: reinsert_eval(T, U, I0, h, p, unit_cost, fixed, consumption[s0:s1],
                                     mean=False, **kw),
        S, batch, bytes_per_scenario=per, device=consumption.device, min_batch=min_batch)
    value = torch.cat([r["value"] for _, _, r in parts]) if parts else \
        torch.empty(0, dtype=torch.float32, device=consumption.device)
    pol = [r["policy"] for _, _, r in parts]
    policy = torch.cat(pol) if parts and pol[0] is not None else None
    return {"value": value, "policy": policy, "mean": value.double().mean() if S else
            torch.zeros((), dtype=torch.float64, device=consumption.device), "batches": sizes}


def status(clear: bool = True) -> int:
    """Synchronise and return the device status bits (FLAG_*)."""
    flags = ctypes.c_uint32(0)
    rc = _load().sdp_device_status(1 if clear else 0, ctypes.byref(flags))
    _check(rc)
    return int(flags.value)


def _split_struct(tour, Q, demands, coords, dist, cost, pred, pred_dtype, algo, mean,
                  warps, ring, overload_penalty=None):
    n = int(tour.numel())
    S = int(demands.shape[0]) if demands.dim() == 2 else (int(demands.numel()) // n if n else 0)
    a = SplitArgs()
    a.n, a.Q, a.S = n, int(Q), S
    a.tour = _dev_ptr(tour, "tour", torch.int32)
    a.coords = _dev_ptr(coords, "coords", torch.float32)
    a.dist = _dev_ptr(dist, "dist", torch.float32)
    a.demands = _demands_ptr(demands)
    a.cost_out = _dev_ptr(cost, "cost")
    a.pred_out = _dev_ptr(pred, "pred")
    a.pred_dtype = pred_dtype
    a.algo = ALGOS[algo]
    a.mean_out = _dev_ptr(mean, "mean")
    a.warps_per_cta = int(warps)
    a.ring = int(ring)
    if overload_penalty is not None:  # soft capacity
        a.capacity_mode = 1
        a.overload_penalty = float(overload_penalty)
    return a


def split_eval(tour, Q, demands, *, coords=None, dist=None, preds=None, algo="auto",
               mean=True, warps=0, ring=0, overload_penalty=None, stream=None):
    """Split of one giant tour over S demand scenarios (Eq. eqdpA).

    tour int32 [n] (permutation of 1..n), demands int32 [S, n] by customer id
    (CUDA, or pinned host memory read by the kernels over the host link),
    coords fp32 [n+1, 2] (node 0 = depot) or dist fp32 [n+1, n+1].
    preds: None, "u16" (returned as int16 holding the uint16 bits) or "i32".
    Returns dict(cost fp32 [S], pred [S, n] or None, mean fp64 0-d tensor or
    None).  overload_penalty (float): soft capacity -- every split allowed,
    that much per unit of route load above Q.  Asynchronous on the current
    stream.
    """
    _load()
    dev = tour.device
    n = int(tour.numel())
    S = int(demands.shape[0])
    cost = torch.empty(S, dtype=torch.float32, device=dev)
    pd = 0
    pred = None
    if preds is not None:
        pd = PRED_DTYPES[preds]
        pred = torch.empty((S, n), dtype=torch.int16 if preds == "u16" else torch.int32,
                           device=dev)
    m = torch.empty((), dtype=torch.float64, device=dev) if mean else None
    a = _split_struct(tour, Q, demands, coords, dist, cost, pred, pd, algo, m, warps, ring,
                      overload_penalty)
    ws = _workspace(_load().sdp_split_workspace_bytes(ctypes.byref(a)), dev)
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    _check(_load().sdp_split_eval(ctypes.byref(a), _stream(stream)))
    return {"cost": cost, "pred": pred, "mean": m}


def split_fleet_eval(tour, Q, demands, max_routes, *, coords=None, dist=None, routes=True,
                     algo="auto", mean=True, stream=None):
    """Fleet-limited Split: at most max_routes routes per scenario (hard
    capacity; the extensive model's fleet-size constraint, Appendix A, on
    the recursion of Eq. eqdpA).  Arguments as split_eval; algo "auto" or "plain".  Returns
    dict(cost fp32 [S] (+inf where no split fits), nroutes int32 [S],
    route uint8 [S, n] (route of each position, 255 when infeasible) or None,
    mean fp64 0-d tensor or None)."""
    _load()
    dev = tour.device
    n = int(tour.numel())
    S = int(demands.shape[0])
    cost = torch.empty(S, dtype=torch.float32, device=dev)
    nroutes = torch.empty(S, dtype=torch.int32, device=dev)
    route = torch.empty((S, n), dtype=torch.uint8, device=dev) if routes else None
    m = torch.empty((), dtype=torch.float64, device=dev) if mean else None
    a = _split_struct(tour, Q, demands, coords, dist, cost, None, 0, algo, m, 0, 0)
    ws = _workspace(_load().sdp_split_fleet_workspace_bytes(ctypes.byref(a), int(max_routes),
                                                            1 if routes else 0), dev)
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    _check(_load().sdp_split_fleet_eval(ctypes.byref(a), int(max_routes),
                                        _dev_ptr(nroutes, "nroutes"), _dev_ptr(route, "route"),
                                        _stream(stream)))
    return {"cost": cost, "nroutes": nroutes, "route": route, "mean": m}


def split_count_arcs(tour, Q, demands, *, coords=None, dist=None, per_scenario=True,
                     stream=None):
    """Capacity-feasible arcs (p, i) of Eq. eqdpA per scenario (int64 [S])
    and their total (uint64 stored in an int64 0-d tensor)."""
    _load()
    dev = tour.device
    S = int(demands.shape[0])
    arcs = torch.empty(S, dtype=torch.int64, device=dev) if per_scenario else None
    total = torch.zeros((), dtype=torch.int64, device=dev)
    a = _split_struct(tour, Q, demands, coords, dist, None, None, 0, "auto", None, 0, 0)
    ws = _workspace(_load().sdp_split_workspace_bytes(ctypes.byref(a)), dev)
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    _check(_load().sdp_split_count_arcs(ctypes.byref(a), _dev_ptr(arcs, "arcs"),
                                        _dev_ptr(total, "total"), _stream(stream)))
    return arcs, total


def split_backward(tour, Q, demands, dist, grad_mean, *, pred=None, pred_dtype=None,
                   algo="auto", want_hist=False, warps=0, ring=0, stream=None):
    """d mean / d dist (fp32 [n+1, n+1]) as scenario-averaged arc-usage counts
    times grad_mean (device fp32 scalar): the route cost W of Sec. 2 is a sum
    of travel costs, so the optimal split's cost is piecewise linear in them.  pred: the forward's predecessors,
    or None to recompute them in the fused forward + backtrack kernel
    (warps / ring: the DEQUE launch shape, as in split_eval; 0 = default)."""
    _load()
    dev = tour.device
    n = int(tour.numel())
    grad = torch.empty((n + 1, n + 1), dtype=torch.float32, device=dev)
    hist = torch.empty(2 * n, dtype=torch.int64, device=dev) if want_hist else None
    pd = 0
    if pred is not None:
        pd = PRED_DTYPES[pred_dtype or ("u16" if pred.element_size() == 2 else "i32")]
    a = _split_struct(tour, Q, demands, None, dist, None, None, pd, algo, None, warps, ring)
    ws = _workspace(_load().sdp_split_backward_workspace_bytes(ctypes.byref(a)), dev)
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    gm = grad_mean.reshape(()).to(device=dev, dtype=torch.float32).contiguous()
    _check(_load().sdp_split_backward(ctypes.byref(a), _dev_ptr(pred, "pred"),
                                      _dev_ptr(gm, "grad_mean"), _dev_ptr(grad, "grad"),
                                      _dev_ptr(hist, "hist"), _stream(stream)))
    return grad, hist


class GraphedSplitBackward:
    """split_backward (fused forward + backtrack) captured once in a CUDA
    graph and replayed: the hist reset, tour preparation, DP kernel, the
    recomputation of flagged scenarios and the gradient assembly go to the
    device as one launch per step, without the per-call host work.

    The graph reads tour, demands, dist and grad_mean where they were at
    capture, so refill those tensors in place between replays (same shapes;
    grad_mean is read in place when it is a CUDA fp32 scalar, else a copy
    taken at construction is used);
    run() returns the same grad (and hist) tensors every time, overwritten
    by each replay.  One warm-up call on a side stream sets up the library's
    per-device state before the capture."""

    def __init__(self, tour, Q, demands, dist, grad_mean, *, want_hist=False):
        _load()
        gm = grad_mean.reshape(()).to(device=tour.device, dtype=torch.float32)
        self._keep = (tour, demands, dist, gm)
        args = (tour, Q, demands, dist, gm)
        side = torch.cuda.Stream(device=tour.device)
        side.wait_stream(torch.cuda.current_stream(tour.device))
        with torch.cuda.stream(side):
            split_backward(*args, want_hist=want_hist)
        torch.cuda.current_stream(tour.device).wait_stream(side)
        torch.cuda.synchronize(tour.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self.grad, self.hist = split_backward(*args, want_hist=want_hist)

    def run(self):
        """Replays the step on the current stream; returns (grad, hist)."""
        self.graph.replay()
        return self.grad, self.hist


class SplitMeanCost(torch.autograd.Function):
    """mean_s J_s(n) (the SAA objective of Sec. 2) as a differentiable
    function of the travel-cost matrix.

    forward(dist [n+1, n+1] fp32 CUDA, tour, demands, Q, keep_pred=False)
    returns the FP64 scenario mean (0-d); backward returns
    d mean / d dist = (1/S) x arc-usage counts of the optimal splits (the
    cost is piecewise linear in dist), computed by the library's backtrack
    kernel from stored predecessors (keep_pred=True) or by the fused
    forward + on-chip backtrack kernel."""

    @staticmethod
    def forward(ctx, dist, tour, demands, Q, keep_pred=False):
        r = split_eval(tour, Q, demands, dist=dist, preds="u16" if keep_pred else None)
        ctx.save_for_backward(dist, tour, demands)
        ctx.Q = int(Q)
        ctx.pred = r["pred"]
        return r["mean"]

    @staticmethod
    def backward(ctx, grad_out):
        dist, tour, demands = ctx.saved_tensors
        pred = ctx.pred
        if pred is not None and pred.dtype != torch.int16:
            pred = pred.view(torch.int16)
        g, _ = split_backward(tour, ctx.Q, demands, dist, grad_out, pred=pred,
                              pred_dtype="u16" if pred is not None else None)
        return g, None, None, None, None


REINSERT_ALGOS = {"auto": 0, "warp": 1, "lane": 2}


def reinsert_eval(T, U, I0, h, p, unit_cost, fixed, consumption, *, table=None,
                  policy=True, value0=False, mean=True, algo="auto", route_cost=None,
                  route_cap=None, stream=None):
    """Backward DP of the OU reinsertion over S scenarios (Algorithm
    SolveBatchDP).  fixed fp32 [T] CUDA, consumption int32 [S, T] CUDA, table
    (optional) fp32 [U+1].  algo: "auto", "warp" (one warp per scenario) or
    "lane" (one lane per scenario).  Route options: route_cost fp32 CUDA
    [T, K] and route_cap int32 CUDA [S, T, K] (fixed may then be None); the
    policy holds 0 (no delivery) or r + 1.  Returns dict(value fp32 [S],
    policy uint8 [S, T], value0 fp32 [S, U+1], mean fp64 0-d)."""
    lib = _load()
    dev = consumption.device
    S = int(consumption.shape[0])
    val = torch.empty(S, dtype=torch.float32, device=dev)
    pol = torch.empty((S, T), dtype=torch.uint8, device=dev) if policy else None
    v0 = torch.empty((S, U + 1), dtype=torch.float32, device=dev) if value0 else None
    m = torch.empty((), dtype=torch.float64, device=dev) if mean else None
    a = ReinsertArgs()
    a.T, a.U, a.I0, a.algo = int(T), int(U), int(I0), REINSERT_ALGOS[algo]
    a.h, a.p, a.unit_cost = float(h), float(p), float(unit_cost)
    a.S = S
    a.fixed = _dev_ptr(fixed, "fixed", torch.float32)
    if route_cost is not None:
        a.n_routes = int(route_cost.shape[-1])
        a.route_cost = _dev_ptr(route_cost, "route_cost", torch.float32)
        a.route_cap = _dev_ptr(route_cap, "route_cap", torch.int32)
    a.end_cost_table = _dev_ptr(table, "table", torch.float32)
    a.consumption = _dev_ptr(consumption, "consumption", torch.int32)
    a.value_out = _dev_ptr(val, "value")
    a.policy_out = _dev_ptr(pol, "policy")
    a.value0_out = _dev_ptr(v0, "value0")
    a.mean_out = _dev_ptr(m, "mean")
    ws = _workspace(lib.sdp_reinsert_workspace_bytes(ctypes.byref(a)), dev)
    a.workspace, a.workspace_bytes = ws.data_ptr(), ws.numel()
    _check(lib.sdp_reinsert_eval(ctypes.byref(a), _stream(stream)))
    return {"value": val, "policy": pol, "value0": v0, "mean": m}


class SplitPlan:
    """Batched Split over B giant tours of uneven length, S scenarios each
    (the candidate evaluations that Tables cand_cvrp / gpu_dsirp count):
    one persistent launch (work queue over (tour, 32-scenario tile) items,
    longest tours first) replayed from a CUDA graph.

    n: int sequence [B]; tours: int32 CUDA [sum n_b] (concatenated
    permutations); coords: fp32 CUDA [sum (n_b+1), 2] (each tour's depot row
    first); demands: int32 CUDA holding tour b's [S, n_b] block at element
    offset dem_off[b] (default: blocks back to back).  Outputs: self.costs
    fp32 [B, S], self.means fp64 [B].
    """

    def __init__(self, n, tours, coords, demands, Q, S, dem_off=None):
        import numpy as np
        lib = _load()
        self._lib = lib
        self.n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
        B = int(self.n.shape[0])
        self.B, self.S, self.Q = B, int(S), int(Q)
        self.tour_off = np.zeros(B, np.int64)
        self.tour_off[1:] = np.cumsum(self.n[:-1], dtype=np.int64)
        self.coord_off = np.zeros(B, np.int64)
        self.coord_off[1:] = np.cumsum(self.n[:-1].astype(np.int64) + 1)
        if dem_off is None:
            dem_off = np.zeros(B, np.int64)
            dem_off[1:] = np.cumsum(self.n[:-1].astype(np.int64) * self.S)
        self.dem_off = np.ascontiguousarray(np.asarray(dem_off, dtype=np.int64))
        dev = demands.device
        self.tours, self.coords, self.demands = tours, coords, demands
        self.costs = torch.empty((B, self.S), dtype=torch.float32, device=dev)
        self.means = torch.empty(B, dtype=torch.float64, device=dev)
        d = BatchDesc()
        d.B, d.Q, d.S = B, self.Q, self.S
        d.n_host = self.n.ctypes.data
        d.tour_off_host = self.tour_off.ctypes.data
        d.tours = _dev_ptr(tours, "tours", torch.int32)
        d.coord_off_host = self.coord_off.ctypes.data
        d.coords = _dev_ptr(coords, "coords", torch.float32)
        d.dem_off_host = self.dem_off.ctypes.data
        d.demands = _dev_ptr(demands, "demands", torch.int32)
        d.costs_out = _dev_ptr(self.costs, "costs")
        d.means_out = _dev_ptr(self.means, "means")
        self._h = ctypes.c_void_p()
        _check(lib.sdp_split_plan_create(ctypes.byref(d), ctypes.byref(self._h)))

    def run(self, stream=None):
        _check(self._lib.sdp_plan_run(self._h, _stream(stream)))
        return self.costs, self.means

    def autotune(self, cache_path=None, stream=None):
        cp = cache_path.encode() if cache_path else None
        _check(self._lib.sdp_plan_autotune(self._h, _stream(stream), cp))
        return self.info()

    def info(self):
        w, r, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        items = ctypes.c_int64()
        ns = ctypes.c_int32()
        _check(self._lib.sdp_plan_info(self._h, ctypes.byref(w), ctypes.byref(r),
                                       ctypes.byref(c), ctypes.byref(items)))
        _check(self._lib.sdp_plan_scenarios_per_lane(self._h, ctypes.byref(ns)))
        return {"warps_per_cta": w.value, "ring": r.value, "ctas": c.value,
                "items": items.value, "scenarios_per_lane": ns.value}

    def configure(self, warps_per_cta, ring=16, scenarios_per_lane=1):
        """Select a launch shape by hand (see sdp_plan_configure)."""
        _check(self._lib.sdp_plan_configure(self._h, int(warps_per_cta), int(ring),
                                            int(scenarios_per_lane)))
        return self.info()

    def kernel_ms(self):
        ms = ctypes.c_float()
        _check(self._lib.sdp_plan_kernel_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def count_arcs(self, stream=None):
        t = ctypes.c_uint64()
        _check(self._lib.sdp_plan_count_arcs(self._h, _stream(stream), ctypes.byref(t)))
        return int(t.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.sdp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MOVES = {"2opt": 1, "relocate": 2, "swap": 4}


class SaaSearch:
    """SAA local search over giant tours (the candidate loop of Sec. "Decision
    Quality under Fixed Time Budgets", with local-search moves in place of the
    paper's genetic algorithm): every iteration scores the current
    tour and B neighbours (2-opt / relocate / swap moves drawn from a
    SplitMix64 stream) by their Split mean over the same scenario set, in one
    batched-plan replay, and keeps the best neighbour if it is strictly
    better.  tour0: int32 CUDA [n]; coords fp32 CUDA [n+1, 2]; demands int32
    CUDA [S, n] (16-byte aligned; shared by every candidate)."""

    def __init__(self, tour0, coords, demands, Q, B, *, seed=0,
                 moves=("2opt", "relocate", "swap")):
        lib = _load()
        self._lib = lib
        self.n = int(tour0.numel())
        self.S = int(demands.shape[0])
        self.B, self.Q = int(B), int(Q)
        self.coords, self.demands = coords, demands  # kept alive for the search
        d = SaaSearchDesc()
        d.n, d.Q, d.S, d.B = self.n, self.Q, self.S, self.B
        d.coords = _dev_ptr(coords, "coords", torch.float32)
        d.demands = _dev_ptr(demands, "demands", torch.int32)
        d.tour0 = _dev_ptr(tour0, "tour0", torch.int32)
        d.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        d.moves = sum(MOVES[m] for m in moves)
        self._dev = demands.device
        self._h = ctypes.c_void_p()
        _check(lib.sdp_saa_search_create(ctypes.byref(d), ctypes.byref(self._h)))

    def run(self, iters, stream=None):
        """(trace fp64 [iters]: best mean after each iteration, accepted int32
        [iters]: neighbour taken or -1), on the device."""
        trace = torch.empty(max(int(iters), 0), dtype=torch.float64, device=self._dev)
        acc = torch.empty(max(int(iters), 0), dtype=torch.int32, device=self._dev)
        _check(self._lib.sdp_saa_search_run(self._h, int(iters), _dev_ptr(trace, "trace"),
                                            _dev_ptr(acc, "accepted"), _stream(stream)))
        return trace, acc

    def state(self, stream=None):
        """(current tour int32 [n], means fp64 [B+1] of the last iteration:
        [0] the tour it started from, [1+k] neighbour k)."""
        tour = torch.empty(self.n, dtype=torch.int32, device=self._dev)
        means = torch.empty(self.B + 1, dtype=torch.float64, device=self._dev)
        _check(self._lib.sdp_saa_search_state(self._h, _dev_ptr(tour, "tour"),
                                              _dev_ptr(means, "means"), _stream(stream)))
        return tour, means

    def count_arcs(self, stream=None):
        """Feasible arcs of every tour the last iteration scored."""
        t = ctypes.c_uint64()
        _check(self._lib.sdp_saa_search_count_arcs(self._h, _stream(stream), ctypes.byref(t)))
        return int(t.value)

    def autotune(self, cache_path=None, stream=None):
        cp = cache_path.encode() if cache_path else None
        _check(self._lib.sdp_saa_search_autotune(self._h, _stream(stream), cp))
        return self.info()

    def info(self):
        """Launch shape of the search's plan (see SplitPlan.info)."""
        w, r, c, ns = (ctypes.c_int32() for _ in range(4))
        _check(self._lib.sdp_saa_search_plan_info(self._h, ctypes.byref(w), ctypes.byref(r),
                                                  ctypes.byref(c), ctypes.byref(ns)))
        return {"warps_per_cta": w.value, "ring": r.value, "ctas": c.value,
                "scenarios_per_lane": ns.value}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.sdp_saa_search_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Plain FP64 CPU oracle for the scenario-batched Bellman updates of
arXiv 2602.05179 (Split for CVRPSD; order-up-to inventory reinsertion).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2602_05179_gb300``) and imports nothing from it;
both sides receive the same seeded input arrays.

The arithmetic lives in ``sdp_oracle.c`` (plain C, FP64, OpenMP over
scenarios); this module only compiles it with gcc and marshals numpy arrays.
Each function cites the passage of the paper it restates; see the C file.

Parity pins (tests/test_oracle_*.py): the three worked examples printed in the
paper (min-plus toy, Split toy, inventory toy), brute-force enumeration of all
splits (n <= 10; with a route limit for the fleet-limited Split) and all
delivery sequences (T <= 8), closed forms (single
route = closed TSP tour when total demand <= Q; one route per customer when
every demand is Q; zero consumption; deliver-every-day), invariants
(monotonicity in Q, in the cost parameters) and central finite differences of
the FP64 mean for the arc-usage gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sdp_oracle.c into liboracle.so (gcc, -O2, OpenMP, no FP
    contraction so every FP64 operation rounds exactly as written)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.oracle_version.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_minplus_matvec.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.oracle_minplus_matvec.restype = None
        lib.oracle_split.argtypes = [ctypes.c_int, P, P, P, i32, i64, P, P, P, P,
                                     P, P, ctypes.c_int]
        lib.oracle_split.restype = ctypes.c_int
        lib.oracle_split_soft.argtypes = [ctypes.c_int, P, P, P, i32, f64, i64, P, P, P, P,
                                          P, P, ctypes.c_int]
        lib.oracle_split_soft.restype = ctypes.c_int
        lib.oracle_split_fleet.argtypes = [ctypes.c_int, P, P, P, i32, ctypes.c_int, i64, P,
                                           P, P, P, P, P, ctypes.c_int]
        lib.oracle_split_fleet.restype = ctypes.c_int
        lib.oracle_reinsert_routes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f64,
                                               f64, f64, ctypes.c_int, P, P, P, i64, P, P, P,
                                               P, P, P, ctypes.c_int]
        lib.oracle_reinsert_routes.restype = ctypes.c_int
        lib.oracle_split_matrix.argtypes = [ctypes.c_int, P, P, P, i32, P, P, P]
        lib.oracle_split_matrix.restype = ctypes.c_int
        lib.oracle_split_route_counts.argtypes = [ctypes.c_int, i64, P, P, P, P]
        lib.oracle_split_route_counts.restype = ctypes.c_int
        lib.oracle_split_mean_grad.argtypes = [ctypes.c_int, P, i64, P, P]
        lib.oracle_split_mean_grad.restype = ctypes.c_int
        lib.oracle_reinsert.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        f64, f64, f64, P, P, i64, P, P, P, P, P,
                                        P, ctypes.c_int]
        lib.oracle_reinsert.restype = ctypes.c_int
        lib.oracle_reinsert_forward.argtypes = [ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, f64, f64, f64, P,
                                                P, P, P, P]
        lib.oracle_reinsert_forward.restype = f64
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def minplus_matvec(A, J):
    """out[j] = min_i A[i, j] + J[i]  (+inf masked); returns (out, argmin)."""
    A = _c(A, np.float64)
    J = _c(J, np.float64)
    m, k = A.shape
    out = np.empty(k, np.float64)
    arg = np.empty(k, np.int32)
    _load().oracle_minplus_matvec(m, k, _ptr(A), _ptr(J), _ptr(out), _ptr(arg))
    return out, arg


def split(tour, Q, demands, coords=None, dist=None, *, want_pred=True,
          want_margin=False, want_arcs=True, nthreads=0):
    """Split DP (Eq. eqdpA) over S scenarios.

    tour: int32 [n], permutation of 1..n.  demands: int32 [S, n] indexed by
    customer id.  Exactly one of coords (float32 [(n+1), 2], row 0 = depot) or
    dist (float32 [(n+1), (n+1)]).  Returns a dict with cost [S] (FP64),
    pred [S, n] int32, margin [S, n], arcs [S] int64 and mean (FP64).
    """
    tour = _c(tour, np.int32)
    n = int(tour.shape[0])
    demands = _c(demands, np.int32)
    if n > 0:
        demands = demands.reshape(-1, n)
    S = int(demands.shape[0]) if demands.ndim == 2 else 0
    coords = _c(coords, np.float32)
    dist = _c(dist, np.float32)
    cost = np.empty(S, np.float64)
    pred = np.empty((S, n), np.int32) if want_pred else None
    margin = np.empty((S, n), np.float64) if want_margin else None
    arcs = np.empty(S, np.int64) if want_arcs else None
    mean = np.zeros(1, np.float64)
    rc = _load().oracle_split(n, _ptr(tour), _ptr(coords), _ptr(dist), int(Q), S,
                              _ptr(demands), _ptr(cost), _ptr(pred), _ptr(margin),
                              _ptr(arcs), _ptr(mean), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_split failed: {rc}")
    return {"cost": cost, "pred": pred, "margin": margin, "arcs": arcs,
            "mean": float(mean[0])}


def split_fleet(tour, Q, K, demands, coords=None, dist=None, *, want_route=True,
                want_margin=False, nthreads=0):
    """Fleet-limited Split: at most K routes (Appendix A, constraint
    eq:fleet_size), hard capacity as in Eq. eqdpA.  Same arguments as split()
    plus K >= 1.  Returns a dict with cost [S] (FP64, +inf where no split into
    at most K routes fits), nroutes [S] int32, route [S, n] int32 (index of the
    route serving each position, -1 when infeasible), margin [S] (relative gap
    to the second-best candidate at the tightest choice of the optimal split)
    and mean."""
    tour = _c(tour, np.int32)
    n = int(tour.shape[0])
    demands = _c(demands, np.int32)
    if n > 0:
        demands = demands.reshape(-1, n)
    S = int(demands.shape[0]) if demands.ndim == 2 else 0
    coords = _c(coords, np.float32)
    dist = _c(dist, np.float32)
    cost = np.empty(S, np.float64)
    nroutes = np.empty(S, np.int32)
    route = np.empty((S, n), np.int32) if want_route else None
    margin = np.empty(S, np.float64) if want_margin else None
    mean = np.zeros(1, np.float64)
    rc = _load().oracle_split_fleet(n, _ptr(tour), _ptr(coords), _ptr(dist), int(Q), int(K), S,
                                    _ptr(demands), _ptr(cost), _ptr(nroutes), _ptr(route),
                                    _ptr(margin), _ptr(mean), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_split_fleet failed: {rc}")
    return {"cost": cost, "nroutes": nroutes, "route": route, "margin": margin,
            "mean": float(mean[0])}


def split_soft(tour, Q, beta, demands, coords=None, dist=None, *, want_pred=True,
               want_margin=False, nthreads=0):
    """Soft-capacity Split (every split allowed, beta per unit of route load
    above Q).  Same arguments and results as split()."""
    tour = _c(tour, np.int32)
    n = int(tour.shape[0])
    demands = _c(demands, np.int32)
    if n > 0:
        demands = demands.reshape(-1, n)
    S = int(demands.shape[0]) if demands.ndim == 2 else 0
    cost = np.empty(S, np.float64)
    pred = np.empty((S, n), np.int32) if want_pred else None
    margin = np.empty((S, n), np.float64) if want_margin else None
    arcs = np.empty(S, np.int64)
    mean = np.zeros(1, np.float64)
    rc = _load().oracle_split_soft(n, _ptr(tour), _ptr(_c(coords, np.float32)),
                                   _ptr(_c(dist, np.float32)), int(Q), float(beta), S,
                                   _ptr(demands), _ptr(cost), _ptr(pred), _ptr(margin),
                                   _ptr(arcs), _ptr(mean), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_split_soft failed: {rc}")
    return {"cost": cost, "pred": pred, "margin": margin, "arcs": arcs,
            "mean": float(mean[0])}


def split_matrix(tour, Q, q_by_customer, coords=None, dist=None):
    """One scenario through the explicit masked matrix A; returns (A, V)."""
    tour = _c(tour, np.int32)
    n = int(tour.shape[0])
    q = _c(q_by_customer, np.int32)
    A = np.empty((n + 1, n + 1), np.float64)
    V = np.empty(n + 1, np.float64)
    rc = _load().oracle_split_matrix(n, _ptr(tour), _ptr(_c(coords, np.float32)),
                                     _ptr(_c(dist, np.float32)), int(Q), _ptr(q),
                                     _ptr(A), _ptr(V))
    if rc != 0:
        raise ValueError(f"oracle_split_matrix failed: {rc}")
    return A, V


def split_route_counts(pred):
    """Route start/end histograms over tour positions from backtracked preds."""
    pred = _c(pred, np.int32)
    S, n = pred.shape
    start = np.empty(n, np.int64)
    end = np.empty(n, np.int64)
    skipped = np.zeros(1, np.int64)
    _load().oracle_split_route_counts(n, S, _ptr(pred), _ptr(start), _ptr(end),
                                      _ptr(skipped))
    return start, end, int(skipped[0])


def split_mean_grad(tour, pred):
    """d mean / d dist as (1/S) x arc-usage counts of the backtracked splits."""
    tour = _c(tour, np.int32)
    pred = _c(pred, np.int32)
    S, n = pred.shape
    g = np.empty((n + 1, n + 1), np.float64)
    _load().oracle_split_mean_grad(n, _ptr(tour), S, _ptr(pred), _ptr(g))
    return g


def reinsert(T, U, I0, h, p, unit_cost, fixed, consumption, H=None, *,
             want_policy=True, want_value0=False, want_margin=False, nthreads=0):
    """Backward DP (Algorithm SolveBatchDP) + backtrack over S scenarios.

    consumption: int32 [S, T]; fixed: float32 [T] (per-day routing cost f_t).
    H (optional float64 [U+1]) switches the end-of-day cost to a table of the
    end inventory.  Returns a dict with value [S], policy [S, T] uint8,
    value0 [S, U+1], margin [S, T, U+1] and mean.
    """
    cons = _c(consumption, np.int32).reshape(-1, T)
    S = int(cons.shape[0])
    fixed = _c(fixed, np.float32)
    H = _c(H, np.float64)
    value = np.empty(S, np.float64)
    policy = np.empty((S, T), np.uint8) if want_policy else None
    value0 = np.empty((S, U + 1), np.float64) if want_value0 else None
    margin = np.empty((S, T, U + 1), np.float64) if want_margin else None
    mean = np.zeros(1, np.float64)
    rc = _load().oracle_reinsert(int(T), int(U), int(I0), float(h), float(p),
                                 float(unit_cost), _ptr(fixed), _ptr(H), S,
                                 _ptr(cons), _ptr(value), _ptr(policy),
                                 _ptr(value0), _ptr(margin), _ptr(mean),
                                 int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_reinsert failed: {rc}")
    return {"value": value, "policy": policy, "value0": value0, "margin": margin,
            "mean": float(mean[0])}


def reinsert_forward(T, U, I0, h, p, unit_cost, fixed, consumption_row, H=None,
                     want_A=False):
    """Forward min-plus recursion (Eq. eqdp2) for ONE scenario.

    Returns (value, Jhist [(T+1), U+1], A [T, U+1, U+1] or None)."""
    fixed = _c(fixed, np.float32)
    cons = _c(consumption_row, np.int32)
    H = _c(H, np.float64)
    A = np.empty((T, U + 1, U + 1), np.float64) if want_A else None
    Jh = np.empty((T + 1, U + 1), np.float64)
    v = _load().oracle_reinsert_forward(int(T), int(U), int(I0), float(h), float(p),
                                        float(unit_cost), _ptr(fixed), _ptr(H),
                                        _ptr(cons), _ptr(A), _ptr(Jh))
    return float(v), Jh, A


def reinsert_routes(T, U, I0, h, p, unit_cost, rcost, cap, consumption, *, H=None,
                    want_value0=False, want_margin=False, nthreads=0):
    """Reinsertion with K route options per day: rcost float32 [T, K] (insertion
    cost of route r on day t), cap int32 [S, T, K] (its residual capacity in
    scenario s; a delivery of U - I rides route r only if cap >= U - I).
    Returns value [S], policy uint8 [S, T] (0 = no delivery, r + 1 = route r),
    optional value0 [S, U+1] and margin [S, T, U+1], and mean."""
    cons = _c(consumption, np.int32).reshape(-1, T)
    S = int(cons.shape[0])
    rcost = _c(rcost, np.float32).reshape(T, -1)
    K = int(rcost.shape[1])
    cap = _c(cap, np.int32).reshape(S, T, K)
    H = _c(H, np.float64)
    value = np.empty(S, np.float64)
    policy = np.empty((S, T), np.uint8)
    value0 = np.empty((S, U + 1), np.float64) if want_value0 else None
    margin = np.empty((S, T, U + 1), np.float64) if want_margin else None
    mean = np.zeros(1, np.float64)
    rc = _load().oracle_reinsert_routes(int(T), int(U), int(I0), float(h), float(p),
                                        float(unit_cost), K, _ptr(rcost), _ptr(cap), _ptr(H),
                                        S, _ptr(cons), _ptr(value), _ptr(policy),
                                        _ptr(value0), _ptr(margin), _ptr(mean), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_reinsert_routes failed: {rc}")
    return {"value": value, "policy": policy, "value0": value0, "margin": margin,
            "mean": float(mean[0])}


from .saa import apply_move, draw_move, saa_search, splitmix64  # noqa: E402,F401

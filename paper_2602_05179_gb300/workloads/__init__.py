"""Seeded synthetic inputs for the scenario-batched Bellman operators.

This module generates inputs only: it holds none of the Split or reinsertion
arithmetic and is the one piece of code that both the CPU oracle's tests and
the CUDA path use.  Every draw is counter based, so any slice of any array
(e.g. a sample of scenarios) can be produced on its own, on the host (numpy,
this file: the reference definition) or on the device (``gen.cu``, checked
bit-for-bit against this file).

Generator (SplitMix64 of Steele, Lea & Flood, 2014, used in counter mode):
    mix(z)  = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
              z *= 0x94D049BB133111EB; z ^= z>>31
    base(seed, stream) = mix(mix(seed + G) + stream * G),   G = 0x9E3779B97F4A7C15
    u(seed, stream, k) = mix(base + (k + 1) * G)            (all mod 2^64)
Distributions:
    uniform int [a, b]       a + u mod (b - a + 1)
    uniform fp32 [a, b)      fp32(a) + fp32(b - a) * (fp32(u >> 40) * 2^-24)
    Poisson(lam) clip [a,b]  inversion: x = (u >> 11) * 2^-53, k = #{j : cdf[j] <= x}
                             with the FP64 CDF table of ``poisson_cdf``; then clip
    permutation of 1..n      1 + stable argsort of u(k), k = 0..n-1

Workloads (sizes and distributions of the paper's experiments; the CVRPLIB and
DSIRP instances are not available, these stand in for them):
    split_c1   n=50,  Q=100, S=1000,  q ~ Poisson(10) clipped [1,Q],  seed 0
    split_c2   n=500, Q=200, S=10^6,  q ~ U{1..30},                   seed 1
    reinsert   T=60,  U=200, I0=100, d ~ Poisson(8), h=1, p=20,
               f_t ~ U[5,50) fp32, S=10^6,                           seed 2
    batch_c4   B=4096 tours, n_b ~ U{20..1000}, Q=150, S=4096 each,
               q ~ Poisson(12) clipped [1,Q],                        seed 3
    adjoint_c5 n=300, full fp32 distance matrix, Q=120, S=10^5,
               q ~ Poisson(10) clipped [1,Q],                        seed 4
Coordinates are uniform fp32 in [0,100)^2 with the depot at (50,50).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

G = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1

# stream ids (fixed: changing them changes every workload)
ST_COORDS, ST_TOUR, ST_DEMAND, ST_CONS, ST_FIXED, ST_NB = 1, 2, 3, 4, 5, 6
ST_RCOST, ST_RCAP = 7, 8  # route-option reinsertion: route costs, residual capacities
ST_BATCH0 = 64  # batched tours: stream = ST_BATCH0 + 4*b + {0: coords, 1: tour, 2: demand}

_U64 = np.uint64


def _mix_int(z: int) -> int:
    z &= MASK
    z ^= z >> 30
    z = (z * M1) & MASK
    z ^= z >> 27
    z = (z * M2) & MASK
    z ^= z >> 31
    return z


def stream_base(seed: int, stream: int) -> int:
    return _mix_int((_mix_int((seed + G) & MASK) + stream * G) & MASK)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z ^ (z >> _U64(30))
        z = z * _U64(M1)
        z = z ^ (z >> _U64(27))
        z = z * _U64(M2)
        z = z ^ (z >> _U64(31))
    return z


def draws(seed: int, stream: int, k0: int, count: int) -> np.ndarray:
    """u(seed, stream, k) for k = k0 .. k0+count-1 as uint64."""
    base = stream_base(seed, stream)
    k = np.arange(k0 + 1, k0 + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _U64(base) + k * _U64(G)
    return _mix(z)


def uniform_int(seed, stream, k0, count, lo, hi) -> np.ndarray:
    u = draws(seed, stream, k0, count)
    span = _U64(hi - lo + 1)
    return (u % span).astype(np.int64).astype(np.int32) + np.int32(lo)


def uniform_f32(seed, stream, k0, count, lo, hi) -> np.ndarray:
    u = draws(seed, stream, k0, count)
    u01 = (u >> _U64(40)).astype(np.float32) * np.float32(2.0 ** -24)
    return np.float32(lo) + np.float32(hi - lo) * u01


def poisson_cdf(lam: float, kmax: int = 255) -> np.ndarray:
    """FP64 CDF table of Poisson(lam), entries k = 0..K (K <= kmax), stopping
    once the CDF reaches 1 - 2^-53 (host libm exp; built once, shared)."""
    out = []
    pmf = math.exp(-lam)
    c = pmf
    out.append(c)
    k = 0
    while c < 1.0 - 2.0 ** -53 and k < kmax:
        k += 1
        pmf = pmf * lam / k
        c = c + pmf
        out.append(c)
    return np.asarray(out, dtype=np.float64)


def poisson_clip(seed, stream, k0, count, lam, lo, hi, cdf=None) -> np.ndarray:
    if cdf is None:
        cdf = poisson_cdf(lam)
    u = draws(seed, stream, k0, count)
    x = (u >> _U64(11)).astype(np.float64) * (2.0 ** -53)
    k = np.searchsorted(cdf, x, side="right").astype(np.int64)
    return np.clip(k, lo, hi).astype(np.int32)


def coords_f32(seed, stream, n) -> np.ndarray:
    """[(n+1), 2] fp32, row 0 = depot (50,50), customers uniform in [0,100)^2."""
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50.0, 50.0)
    if n:
        u = draws(seed, stream, 0, 2 * n)
        u01 = (u >> _U64(40)).astype(np.float32) * np.float32(2.0 ** -24)
        xy[1:] = (u01 * np.float32(100.0)).reshape(n, 2)
    return xy


def permutation(seed, stream, n) -> np.ndarray:
    """Random giant tour: permutation of 1..n (int32)."""
    u = draws(seed, stream, 0, n)
    return (np.argsort(u, kind="stable") + 1).astype(np.int32)


def dist_matrix_f32(coords: np.ndarray) -> np.ndarray:
    """Full (n+1)x(n+1) fp32 Euclidean matrix (FP64 distance, rounded)."""
    c = coords.astype(np.float64)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    return d.astype(np.float32)


# --------------------------------------------------------------------------
@dataclass
class SplitSpec:
    name: str
    n: int
    Q: int
    S: int
    seed: int
    demand: str          # "poisson" | "uniform"
    lam: float = 0.0
    lo: int = 1
    hi: int = 1
    dist_mode: bool = False


SPLIT_C1 = SplitSpec("split_n50_S1e3", 50, 100, 1000, 0, "poisson", lam=10.0, lo=1, hi=100)
SPLIT_C2 = SplitSpec("split_n500_S1e6", 500, 200, 1_000_000, 1, "uniform", lo=1, hi=30)
ADJOINT_C5 = SplitSpec("adjoint_n300_S1e5", 300, 120, 100_000, 4, "poisson", lam=10.0,
                       lo=1, hi=120, dist_mode=True)
# SAA candidate search: one CVRPSD instance (n = 100 customers, Q = 100,
# Poisson(10) demands, 10^4 scenarios), 1024 neighbours per iteration
SAA_C6 = SplitSpec("saa_n100_S1e4", 100, 100, 10_000, 6, "poisson", lam=10.0, lo=1, hi=100)
SAA_B = 1024


def split_tour(spec: SplitSpec):
    """(tour [n] int32, coords [(n+1),2] fp32, dist or None)."""
    tour = permutation(spec.seed, ST_TOUR, spec.n)
    xy = coords_f32(spec.seed, ST_COORDS, spec.n)
    dist = dist_matrix_f32(xy) if spec.dist_mode else None
    return tour, xy, dist


def split_demands(spec: SplitSpec, s0: int = 0, s1: int | None = None) -> np.ndarray:
    """Rows s0..s1-1 of the demand matrix [S, n] (int32, by customer id)."""
    s1 = spec.S if s1 is None else s1
    cnt = (s1 - s0) * spec.n
    k0 = s0 * spec.n
    if spec.demand == "uniform":
        q = uniform_int(spec.seed, ST_DEMAND, k0, cnt, spec.lo, spec.hi)
    else:
        q = poisson_clip(spec.seed, ST_DEMAND, k0, cnt, spec.lam, spec.lo, spec.hi)
    return q.reshape(s1 - s0, spec.n)


@dataclass
class ReinsertSpec:
    name: str
    T: int
    U: int
    I0: int
    h: float
    p: float
    unit_cost: float
    S: int
    seed: int
    lam: float
    f_lo: float
    f_hi: float


REINSERT_C3 = ReinsertSpec("reinsert_T60_U200_S1e6", 60, 200, 100, 1.0, 20.0, 0.0,
                           1_000_000, 2, 8.0, 5.0, 50.0)


def reinsert_fixed(spec: ReinsertSpec) -> np.ndarray:
    return uniform_f32(spec.seed, ST_FIXED, 0, spec.T, spec.f_lo, spec.f_hi)


def reinsert_consumption(spec: ReinsertSpec, s0: int = 0, s1: int | None = None):
    """Rows s0..s1-1 of consumption [S, T] (int32), Poisson(lam), clipped at
    the table's end (no lower clip: zero consumption is a valid day)."""
    s1 = spec.S if s1 is None else s1
    q = poisson_clip(spec.seed, ST_CONS, s0 * spec.T, (s1 - s0) * spec.T, spec.lam,
                     0, 1 << 30)
    return q.reshape(s1 - s0, spec.T)


# Route-option reinsertion: the reinsertion workload with K routes per day;
# route r on day t costs U[5,50) fp32 (shared by the scenarios) and has a
# residual capacity U{0..250} in each scenario (it carries a refill of q only
# if the capacity is at least q).
REINSERT_ROUTES = ReinsertSpec("reinsert_routes_T60_U200_K4_S1e6", 60, 200, 100, 1.0, 20.0, 0.0,
                               1_000_000, 5, 8.0, 5.0, 50.0)
ROUTES_K, ROUTES_CAP_LO, ROUTES_CAP_HI = 4, 0, 250


def reinsert_route_costs(spec: ReinsertSpec, K: int = ROUTES_K) -> np.ndarray:
    return uniform_f32(spec.seed, ST_RCOST, 0, spec.T * K, spec.f_lo, spec.f_hi).reshape(spec.T, K)


def reinsert_route_caps(spec: ReinsertSpec, s0: int = 0, s1: int | None = None,
                        K: int = ROUTES_K) -> np.ndarray:
    """Rows s0..s1-1 of the residual capacities [S, T, K] (int32)."""
    s1 = spec.S if s1 is None else s1
    c = uniform_int(spec.seed, ST_RCAP, s0 * spec.T * K, (s1 - s0) * spec.T * K,
                    ROUTES_CAP_LO, ROUTES_CAP_HI)
    return c.reshape(s1 - s0, spec.T, K)


@dataclass
class BatchSpec:
    name: str
    B: int
    n_lo: int
    n_hi: int
    Q: int
    S: int
    seed: int
    lam: float


BATCH_C4 = BatchSpec("batch_B4096_n20-1000_S4096", 4096, 20, 1000, 150, 4096, 3, 12.0)


def batch_sizes(spec: BatchSpec) -> np.ndarray:
    return uniform_int(spec.seed, ST_NB, 0, spec.B, spec.n_lo, spec.n_hi)


def batch_tour(spec: BatchSpec, b: int, n_b: int):
    st = ST_BATCH0 + 4 * b
    return permutation(spec.seed, st + 1, n_b), coords_f32(spec.seed, st, n_b)


def batch_demands(spec: BatchSpec, b: int, n_b: int, s0: int = 0, s1: int | None = None):
    s1 = spec.S if s1 is None else s1
    st = ST_BATCH0 + 4 * b + 2
    q = poisson_clip(spec.seed, st, s0 * n_b, (s1 - s0) * n_b, spec.lam, 1, spec.Q)
    return q.reshape(s1 - s0, n_b)


# --------------------------------------------------------------------------
# Device twin (gen.cu, libsdpgen.so): the same counter-mode draws written
# straight into CUDA tensors, for inputs too large to build on the host.
_GEN = None


def _gen():
    global _GEN
    if _GEN is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "libsdpgen.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        u64, i64, i32, P = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.sdpgen_uniform_int.argtypes = [u64, u64, i64, i64, i32, i32, P, P]
        lib.sdpgen_uniform_int.restype = ctypes.c_int
        lib.sdpgen_poisson_clip.argtypes = [u64, u64, i64, i64, P, ctypes.c_int, i32, i32, P, P]
        lib.sdpgen_poisson_clip.restype = ctypes.c_int
        _GEN = lib
    return _GEN


def _dev_out(out):
    import torch
    assert out.is_cuda and out.dtype == torch.int32 and out.is_contiguous()
    return out.data_ptr(), torch.cuda.current_stream().cuda_stream


def device_uniform_int(out, seed, stream, k0, lo, hi):
    ptr, st = _dev_out(out)
    rc = _gen().sdpgen_uniform_int(seed, stream, k0, out.numel(), lo, hi, ptr, st)
    if rc != 0:
        raise RuntimeError(f"sdpgen_uniform_int failed: {rc}")
    return out


def device_poisson_clip(out, seed, stream, k0, lam, lo, hi):
    import torch
    cdf = torch.from_numpy(poisson_cdf(lam)).to(out.device)
    ptr, st = _dev_out(out)
    rc = _gen().sdpgen_poisson_clip(seed, stream, k0, out.numel(), cdf.data_ptr(),
                                    int(cdf.numel()), lo, hi, ptr, st)
    if rc != 0:
        raise RuntimeError(f"sdpgen_poisson_clip failed: {rc}")
    torch.cuda.current_stream().synchronize()  # keep cdf alive until the kernel ran
    return out


def split_demands_device(spec: SplitSpec, device="cuda", s0=0, s1=None):
    """Rows s0..s1-1 of the demand matrix generated on the device."""
    import torch
    s1 = spec.S if s1 is None else s1
    out = torch.empty((s1 - s0, spec.n), dtype=torch.int32, device=device)
    if spec.demand == "uniform":
        return device_uniform_int(out, spec.seed, ST_DEMAND, s0 * spec.n, spec.lo, spec.hi)
    return device_poisson_clip(out, spec.seed, ST_DEMAND, s0 * spec.n, spec.lam, spec.lo, spec.hi)


def reinsert_consumption_device(spec: ReinsertSpec, device="cuda", s0=0, s1=None):
    import torch
    s1 = spec.S if s1 is None else s1
    out = torch.empty((s1 - s0, spec.T), dtype=torch.int32, device=device)
    return device_poisson_clip(out, spec.seed, ST_CONS, s0 * spec.T, spec.lam, 0, 1 << 30)


def batch_demands_device(spec: BatchSpec, b: int, n_b: int, out):
    """Fill out (int32 [S, n_b] CUDA view) with tour b's demands."""
    st = ST_BATCH0 + 4 * b + 2
    return device_poisson_clip(out, spec.seed, st, 0, spec.lam, 1, spec.Q)


def reinsert_route_caps_device(spec: ReinsertSpec, device="cuda", s0=0, s1=None,
                               K: int = ROUTES_K):
    import torch
    s1 = spec.S if s1 is None else s1
    out = torch.empty((s1 - s0, spec.T, K), dtype=torch.int32, device=device)
    return device_uniform_int(out, spec.seed, ST_RCAP, s0 * spec.T * K, ROUTES_CAP_LO,
                              ROUTES_CAP_HI)

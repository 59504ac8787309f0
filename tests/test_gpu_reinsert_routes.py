"""GPU parity of the route-option reinsertion (K candidate routes per day;
a delivery rides the cheapest route whose residual capacity holds it)
against the FP64 oracle and the two-action kernel, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.gpu_util import check_reinsert

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _routes_policy_check(gp, orc, cons, U, I0):
    """Policies along the oracle's path, where the decision is unique."""
    op = orc["policy"]
    mg = orc["margin"]
    S, T = op.shape
    checked = 0
    for s in range(S):
        I = I0
        for t in range(T):
            if mg[s, t, I] > 1e-4:
                assert gp[s, t] == op[s, t], (s, t, I)
                checked += 1
            elif gp[s, t] != op[s, t]:
                break
            I = max(0, (U if op[s, t] else I) - int(cons[s, t]))
    return checked


@pytest.mark.parametrize("case", [
    # seed, T, U, I0, S, K, lam, unit_cost, cap_lo, cap_hi
    (0, 12, 20, 10, 100, 1, 4.0, 0.0, 0, 20),
    (1, 30, 31, 0, 65, 3, 9.0, 0.7, 0, 40),    # U + 1 = 32
    (2, 40, 200, 100, 70, 4, 8.0, 0.0, 0, 250),  # the route workload's shape
    (3, 25, 120, 17, 40, 5, 50.0, 0.2, 60, 130),  # consumption above 32 (slow path)
    (4, 20, 0, 0, 33, 2, 3.0, 0.0, 0, 5),      # U = 0: nothing to deliver
    (5, 8, 255, 255, 37, 8, 20.0, 1.5, 100, 255),  # the largest U, I0 = U
])
@pytest.mark.parametrize("algo", ["warp", "lane"])
def test_routes_vs_oracle(case, algo):
    seed, T, U, I0, S, K, lam, c, clo, chi = case
    rng = np.random.default_rng(seed)
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    rcost = rng.uniform(5, 50, (T, K)).astype(np.float32)
    cap = rng.integers(clo, chi + 1, size=(S, T, K)).astype(np.int32)
    o = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, c, rcost, cap, cons, want_value0=True,
                               want_margin=True)
    r = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), value0=True,
                            route_cost=_cuda(rcost), route_cap=_cuda(cap), algo=algo)
    torch.cuda.synchronize()
    check_reinsert(r["value"], None, o, cons, U, I0)
    np.testing.assert_allclose(r["value0"].cpu().double().numpy(), o["value0"], rtol=1e-5,
                               atol=1e-6)
    _routes_policy_check(r["policy"].cpu().numpy(), o, cons, U, I0)
    assert abs(float(r["mean"]) - o["mean"]) <= 1e-5 * max(1.0, abs(o["mean"]))


def test_one_roomy_route_is_the_two_action_kernel():
    """K = 1, capacity U every day, cost fixed[t]: the same FP32 operations as
    the two-action kernel, bit for bit."""
    rng = np.random.default_rng(3)
    S, T, U, I0 = 300, 40, 150, 60
    cons = rng.poisson(9.0, size=(S, T)).astype(np.int32)
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    cap = np.full((S, T, 1), U, np.int32)
    for c in (0.0, 0.4):
        a = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, _cuda(fixed), _cuda(cons), value0=True,
                                algo="warp")
        b = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), value0=True,
                                route_cost=_cuda(fixed[:, None]), route_cap=_cuda(cap))
        torch.cuda.synchronize()
        for key in ("value", "value0", "policy"):
            assert torch.equal(a[key], b[key]), key


@pytest.mark.parametrize("case", [
    # seed, T, U, I0, S, K, lam, unit_cost, cap_lo, cap_hi
    (11, 60, 200, 100, 1000, 4, 8.0, 0.0, 0, 250),   # the route workload's shape
    (12, 17, 90, 33, 97, 1, 6.0, 0.5, 0, 120),       # one route, ragged S
    (13, 33, 63, 5, 64, 7, 15.0, 0.0, -5, 80),       # negative capacities (never usable)
    (14, 12, 255, 0, 40, 8, 40.0, 2.0, 0, 300),      # the largest U, consumption above 32
    (15, 5, 31, 31, 33, 3, 2.0, 0.0, 0, 31),         # U + 1 = 32, I0 = U
])
def test_routes_lane_bit_identical_to_warp(case):
    """The lane kernel's route minimum does the warp kernel's FP32 operations:
    values, C_0 tables and policies (r + 1 of the route taken) are the same."""
    seed, T, U, I0, S, K, lam, c, clo, chi = case
    rng = np.random.default_rng(seed)
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    rcost = rng.uniform(5, 50, (T, K)).astype(np.float32)
    cap = rng.integers(clo, chi + 1, size=(S, T, K)).astype(np.int32)
    kw = dict(value0=True, route_cost=_cuda(rcost), route_cap=_cuda(cap))
    w = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), algo="warp", **kw)
    ln = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), algo="lane", **kw)
    au = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), **kw)
    torch.cuda.synchronize()
    for key in ("value", "value0", "policy"):
        assert torch.equal(w[key], ln[key]), key
        assert torch.equal(au[key], ln[key]), key
    assert float(w["mean"]) == float(ln["mean"])


def test_routes_rejections():
    api = sdp()
    cons = torch.ones((4, 10), dtype=torch.int32, device="cuda")
    rc = torch.ones((10, 2), dtype=torch.float32, device="cuda")
    cap = torch.ones((4, 10, 2), dtype=torch.int32, device="cuda")
    tab = torch.ones(11, dtype=torch.float32, device="cuda")
    for kw, U, code in ((dict(table=tab), 10, -5), ({}, 300, -5)):
        with pytest.raises(api.SdpError) as e:
            api.reinsert_eval(10, U, 0, 1.0, 1.0, 0.0, None, cons, route_cost=rc, route_cap=cap,
                              **kw)
        assert e.value.code == code
    # the lane kernel takes up to 8 route options; AUTO runs more on the warp kernel
    rc9 = torch.ones((10, 9), dtype=torch.float32, device="cuda")
    cap9 = torch.ones((4, 10, 9), dtype=torch.int32, device="cuda")
    with pytest.raises(api.SdpError) as e:
        api.reinsert_eval(10, 10, 0, 1.0, 1.0, 0.0, None, cons, route_cost=rc9, route_cap=cap9,
                          algo="lane")
    assert e.value.code == -5
    r = api.reinsert_eval(10, 10, 0, 1.0, 1.0, 0.0, None, cons, route_cost=rc9, route_cap=cap9)
    torch.cuda.synchronize()
    assert torch.isfinite(r["value"]).all()


def test_routes_full_size_sampled():
    """T=60, U=200, K=4 routes, S=10^6 on the device; sampled scenarios vs
    the oracle."""
    spec = wl.REINSERT_ROUTES
    cons_d = wl.reinsert_consumption_device(spec)
    cap_d = wl.reinsert_route_caps_device(spec)
    np.testing.assert_array_equal(cap_d[5000:5004].cpu().numpy(),
                                  wl.reinsert_route_caps(spec, 5000, 5004))
    rcost = wl.reinsert_route_costs(spec)
    r = sdp().reinsert_eval(spec.T, spec.U, spec.I0, spec.h, spec.p, spec.unit_cost, None,
                            cons_d, route_cost=_cuda(rcost), route_cap=cap_d)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(spec.S, 800, replace=False))
    rows = np.concatenate([rows, [0, spec.S - 1]])
    cons = np.concatenate([wl.reinsert_consumption(spec, int(s), int(s) + 1) for s in rows])
    cap = np.concatenate([wl.reinsert_route_caps(spec, int(s), int(s) + 1) for s in rows])
    o = oracle.reinsert_routes(spec.T, spec.U, spec.I0, spec.h, spec.p, spec.unit_cost, rcost,
                               cap, cons, want_margin=True)
    check_reinsert(r["value"], None, o, cons, spec.U, spec.I0, rows=rows)
    checked = _routes_policy_check(r["policy"].cpu().numpy()[rows], o, cons, spec.U, spec.I0)
    assert checked > 0.8 * len(rows) * spec.T

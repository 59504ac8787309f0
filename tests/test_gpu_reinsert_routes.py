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
def test_routes_vs_oracle(case):
    seed, T, U, I0, S, K, lam, c, clo, chi = case
    rng = np.random.default_rng(seed)
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    rcost = rng.uniform(5, 50, (T, K)).astype(np.float32)
    cap = rng.integers(clo, chi + 1, size=(S, T, K)).astype(np.int32)
    o = oracle.reinsert_routes(T, U, I0, 1.0, 20.0, c, rcost, cap, cons, want_value0=True,
                               want_margin=True)
    r = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, None, _cuda(cons), value0=True,
                            route_cost=_cuda(rcost), route_cap=_cuda(cap))
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


def test_routes_rejections():
    api = sdp()
    cons = torch.ones((4, 10), dtype=torch.int32, device="cuda")
    rc = torch.ones((10, 2), dtype=torch.float32, device="cuda")
    cap = torch.ones((4, 10, 2), dtype=torch.int32, device="cuda")
    tab = torch.ones(11, dtype=torch.float32, device="cuda")
    for kw, U, code in ((dict(algo="lane"), 10, -5), (dict(table=tab), 10, -5), ({}, 300, -5)):
        with pytest.raises(api.SdpError) as e:
            api.reinsert_eval(10, U, 0, 1.0, 1.0, 0.0, None, cons, route_cost=rc, route_cap=cap,
                              **kw)
        assert e.value.code == code


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

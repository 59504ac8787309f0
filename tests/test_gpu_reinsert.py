"""GPU parity of the reinsertion kernels (one scenario per warp, one per
lane) against the FP64 oracle (backward DP of Algorithm SolveBatchDP) and
against each other, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl
from tests.golden_io import arr, load
from tests.gpu_util import check_reinsert

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sdp():
    from paper_2602_05179_gb300 import api
    return api


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("algo", ["warp", "lane"])
def test_reinsert_paper_toy(algo):
    g = load("inventory_toy.json")
    T, U, I0 = g["T"], g["U"], g["I0"]
    table = np.asarray(g["end_cost_table"], np.float32)
    cons = arr(g["consumption"], np.int32)[None, :]
    fixed = np.zeros(T, np.float32)
    r = sdp().reinsert_eval(T, U, I0, 0.0, 0.0, 1.0, _cuda(fixed), _cuda(cons),
                            table=_cuda(table), value0=True, algo=algo)
    torch.cuda.synchronize()
    assert float(r["value"][0]) == g["value"]
    assert r["policy"][0].tolist() == g["policy"]
    # C_0(I) for I = 0, 1, 2 from the oracle's backward DP
    o = oracle.reinsert(T, U, I0, 0.0, 0.0, 1.0, fixed, cons, H=table.astype(np.float64),
                        want_value0=True)
    np.testing.assert_array_equal(r["value0"][0].cpu().numpy(), o["value0"][0])
    assert float(r["mean"]) == g["value"]


@pytest.mark.parametrize("algo", ["auto", "warp", "lane"])
@pytest.mark.parametrize("case", [
    # seed, T, U, I0, S, lam, table, unit_cost
    (0, 8, 12, 5, 100, 4.0, False, 0.0),
    (1, 30, 31, 0, 65, 9.0, False, 0.7),     # U+1 = 32: one register per lane
    (2, 20, 200, 100, 70, 8.0, True, 0.0),    # table mode
    (3, 25, 300, 17, 40, 50.0, False, 0.2),   # KC = 16; consumption > 32 (slow path)
    (4, 60, 0, 0, 33, 3.0, False, 0.0),       # U = 0
    (5, 1, 50, 50, 37, 20.0, False, 1.5),     # T = 1, I0 = U
    (6, 64, 255, 9, 70, 40.0, False, 0.0),    # the largest lane-kernel shape, d > 32
    (7, 40, 100, 60, 200, 8.0, False, 0.0),   # 200 = 6 tiles + 8 rows
    (8, 12, 70, 3, 50, 90.0, True, 0.4),      # table + unit cost, d > U
])
def test_reinsert_cases(case, algo):
    seed, T, U, I0, S, lam, use_table, c = case
    if algo == "lane" and U > 255:
        pytest.skip("the one-scenario-per-lane kernel takes U <= 255")
    rng = np.random.default_rng(seed)
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    table = rng.uniform(0, 30, U + 1).astype(np.float32) if use_table else None
    o = oracle.reinsert(T, U, I0, 1.0, 20.0, c, fixed, cons,
                        H=None if table is None else table.astype(np.float64),
                        want_value0=True, want_margin=True)
    r = sdp().reinsert_eval(T, U, I0, 1.0, 20.0, c, _cuda(fixed), _cuda(cons),
                            table=None if table is None else _cuda(table), value0=True,
                            algo=algo)
    torch.cuda.synchronize()
    check_reinsert(r["value"], r["policy"], o, cons, U, I0)
    v0 = r["value0"].cpu().double().numpy()
    np.testing.assert_allclose(v0, o["value0"], rtol=1e-5, atol=1e-6)
    assert abs(float(r["mean"]) - o["mean"]) <= 1e-5 * max(1.0, abs(o["mean"]))


def test_reinsert_c3_full_size_sampled():
    """T=60, U=200, S=10^6 on the device; sampled scenarios vs the oracle."""
    spec = wl.REINSERT_C3
    cons_d = wl.reinsert_consumption_device(spec)
    np.testing.assert_array_equal(cons_d[777_000:777_020].cpu().numpy(),
                                  wl.reinsert_consumption(spec, 777_000, 777_020))
    fixed = wl.reinsert_fixed(spec)
    r = sdp().reinsert_eval(spec.T, spec.U, spec.I0, spec.h, spec.p, spec.unit_cost,
                            _cuda(fixed), cons_d)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(spec.S, 1500, replace=False))
    rows = np.concatenate([rows, [0, spec.S - 1]])
    cons = np.concatenate([wl.reinsert_consumption(spec, int(s), int(s) + 1) for s in rows])
    o = oracle.reinsert(spec.T, spec.U, spec.I0, spec.h, spec.p, spec.unit_cost, fixed, cons,
                        want_margin=True)
    checked = check_reinsert(r["value"], r["policy"], o, cons, spec.U, spec.I0, rows=rows)
    assert checked > 0.9 * len(rows) * spec.T
    host_mean = r["value"].double().mean().item()
    assert abs(float(r["mean"]) - host_mean) <= 1e-12 * host_mean


@pytest.mark.parametrize("T,U,lam,table,c", [(60, 200, 8.0, False, 0.0), (33, 100, 30.0, False, 0.3),
                                             (64, 255, 12.0, True, 0.0), (5, 31, 2.0, False, 0.0)])
def test_reinsert_lane_and_warp_bit_identical(T, U, lam, table, c):
    """The two mappings evaluate the same FP32 operations in the same order:
    values, C_0 tables and policies agree bit for bit."""
    rng = np.random.default_rng(T * 1000 + U)
    S = 333
    cons = rng.poisson(lam, size=(S, T)).astype(np.int32)
    cons[5, :] = 0
    cons[6, :] = 400  # every day empties the stock
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    tab = _cuda(rng.uniform(0, 30, U + 1).astype(np.float32)) if table else None
    out = {algo: sdp().reinsert_eval(T, U, U // 2, 1.0, 20.0, c, _cuda(fixed), _cuda(cons),
                                     table=tab, value0=True, algo=algo)
           for algo in ("warp", "lane")}
    torch.cuda.synchronize()
    for key in ("value", "policy", "value0"):
        assert torch.equal(out["warp"][key], out["lane"][key]), key


def test_reinsert_lane_rejects_unsupported_shapes():
    fixed = torch.ones(10, dtype=torch.float32, device="cuda")
    cons = torch.ones((4, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(sdp().SdpError) as e:
        sdp().reinsert_eval(10, 256, 0, 1.0, 1.0, 0.0, fixed, cons, algo="lane")
    assert e.value.code == -5
    # a shape both kernels take, without a policy (no decision scratch)
    r = sdp().reinsert_eval(10, 255, 3, 1.0, 1.0, 0.0, fixed, cons, algo="lane", policy=False)
    w = sdp().reinsert_eval(10, 255, 3, 1.0, 1.0, 0.0, fixed, cons, algo="warp", policy=False)
    torch.cuda.synchronize()
    assert torch.equal(r["value"], w["value"])

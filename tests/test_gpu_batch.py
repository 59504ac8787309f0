"""GPU parity of the batched Split plan (persistent kernel + CUDA graph +
autotuned launch shape) against the FP64 oracle and the eager kernels."""
import os

import numpy as np
import pytest

import oracle
from paper_2602_05179_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def api():
    from paper_2602_05179_gb300 import api as a
    return a


def _batch(seed, B, S, Q, nlo, nhi, qhi, n_first=0):
    rng = np.random.default_rng(seed)
    n = rng.integers(nlo, nhi + 1, size=B).astype(np.int32)
    if n_first:
        n[0] = n_first
    tours, coords, dem = [], [], []
    for b in range(B):
        tours.append((rng.permutation(n[b]) + 1).astype(np.int32))
        xy = np.empty((n[b] + 1, 2), np.float32)
        xy[0] = (50, 50)
        xy[1:] = rng.uniform(0, 100, (n[b], 2)).astype(np.float32)
        coords.append(xy)
        dem.append(rng.integers(1, qhi + 1, size=(S, n[b])).astype(np.int32))
    return n, tours, coords, dem


def _plan(n, tours, coords, dem, Q, S):
    t = torch.from_numpy(np.concatenate(tours)).cuda()
    c = torch.from_numpy(np.concatenate(coords)).cuda()
    d = torch.from_numpy(np.concatenate([x.reshape(-1) for x in dem])).cuda()
    return api().SplitPlan(n, t, c, d, Q, S), (t, c, d)


@pytest.mark.parametrize("Q,qhi", [(150, 40), (400, 90)])
def test_batch_small_vs_oracle_and_eager(Q, qhi, tmp_path):
    B, S = 37, 100
    n, tours, coords, dem = _batch(11 + Q, B, S, Q, 1, 300, qhi)
    plan, keep = _plan(n, tours, coords, dem, Q, S)
    assert plan.info()["warps_per_cta"] == -2         # default: the pipelined kernel
    costs, means = plan.run()
    torch.cuda.synchronize()
    c1 = costs.clone()
    for b in range(B):
        o = oracle.split(tours[b], Q, dem[b], coords=coords[b])
        g = costs[b].cpu().double().numpy()
        rel = np.abs(g - o["cost"]) / o["cost"]
        assert rel.max() <= 1e-5, (b, rel.max())
        assert abs(float(means[b]) - o["mean"]) <= 1e-5 * o["mean"]
        # same bits as the eager single-tour call
        r = api().split_eval(torch.from_numpy(tours[b]).cuda(), Q,
                             torch.from_numpy(dem[b]).cuda(),
                             coords=torch.from_numpy(coords[b]).cuda(), algo="deque")
        assert torch.equal(r["cost"], costs[b])
    # graph replay, then autotune (+ cache) give the same bits
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(costs, c1)
    cache = str(tmp_path / "tune.txt")
    info = plan.autotune(cache)
    assert info["warps_per_cta"] in (-2, -1, 0, 1, 2, 4, 8) and info["ring"] in (8, 16)
    assert info["scenarios_per_lane"] in (1, 2)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(costs, c1)
    assert os.path.exists(cache)
    assert plan.autotune(cache) == info   # cache hit
    arcs = plan.count_arcs()
    assert arcs == sum(int(oracle.split(tours[b], Q, dem[b], coords=coords[b])["arcs"].sum())
                       for b in range(B))
    assert plan.kernel_ms() > 0
    assert api().status() & api().FLAG_INFEASIBLE == 0
    plan.close()


@pytest.mark.parametrize("Q,qhi", [(150, 40), (600, 90)])
def test_batch_stream_and_deque_plans_bit_identical(Q, qhi):
    """The streaming plan kernel and the DEQUE batched kernel (forced by
    demand blocks that do not start on 16 bytes) give the same bits, on tours
    shorter and longer than a tensor-memory row, with a ragged last tile
    (S = 164: 5 tiles + 4 rows, every offset a multiple of 4) and a few
    demands above Q."""
    B, S = 29, 164
    # one tour above 1024 customers: the pipelined kernel does not apply
    n, tours, coords, dem = _batch(77 + Q, B, S, Q, 1, 1100, qhi, n_first=1100)
    dem[3][7, 0] = Q + 1
    plan_s, keep_s = _plan(n, tours, coords, dem, Q, S)
    assert plan_s.info()["warps_per_cta"] == -1
    # the same blocks, each one element further along: offsets not multiples of 4
    off = np.zeros(B, np.int64)
    off[1:] = np.cumsum(n[:-1].astype(np.int64) * S)
    off = off + np.arange(1, B + 1)
    buf = torch.zeros(int(off[-1] + n[-1] * S), dtype=torch.int32, device="cuda")
    for b in range(B):
        buf[off[b]:off[b] + n[b] * S] = torch.from_numpy(dem[b].reshape(-1)).cuda()
    t, c, _ = keep_s
    plan_d = api().SplitPlan(n, t, c, buf, Q, S, dem_off=off)
    assert plan_d.info()["warps_per_cta"] >= 0
    cs, ms = plan_s.run()
    cd, md = plan_d.run()
    torch.cuda.synchronize()
    assert torch.equal(cs, cd)
    assert torch.equal(ms.isinf(), md.isinf())
    fin = ~ms.isinf()
    assert torch.equal(ms[fin], md[fin])
    assert api().status() & api().FLAG_INFEASIBLE
    plan_s.close()
    plan_d.close()


@pytest.mark.parametrize("Q,qhi", [(150, 40), (600, 90)])
def test_batch_pipe_and_deque_plans_bit_identical(Q, qhi):
    """The pipelined plan kernel (every tour n <= 1024) and the DEQUE batched
    kernel (forced by demand blocks that do not start on 16 bytes) give the
    same bits on tours shorter and longer than a tensor-memory row, with a
    ragged last tile (S = 164) and a few demands above Q."""
    B, S = 31, 164
    n, tours, coords, dem = _batch(91 + Q, B, S, Q, 1, 1024, qhi)
    dem[5][9, 0] = Q + 1
    plan_p, keep_p = _plan(n, tours, coords, dem, Q, S)
    assert plan_p.info()["warps_per_cta"] == -2
    off = np.zeros(B, np.int64)
    off[1:] = np.cumsum(n[:-1].astype(np.int64) * S)
    off = off + np.arange(1, B + 1)
    buf = torch.zeros(int(off[-1] + n[-1] * S), dtype=torch.int32, device="cuda")
    for b in range(B):
        buf[off[b]:off[b] + n[b] * S] = torch.from_numpy(dem[b].reshape(-1)).cuda()
    t, c, _ = keep_p
    plan_d = api().SplitPlan(n, t, c, buf, Q, S, dem_off=off)
    assert plan_d.info()["warps_per_cta"] >= 0
    cp, mp = plan_p.run()
    cd, md = plan_d.run()
    torch.cuda.synchronize()
    assert torch.equal(cp, cd)
    assert torch.equal(mp.isinf(), md.isinf())
    fin = ~mp.isinf()
    assert torch.equal(mp[fin], md[fin])
    assert api().status() & api().FLAG_INFEASIBLE
    plan_p.close()
    plan_d.close()


@pytest.mark.parametrize("Q,qhi", [(150, 40), (600, 90)])
def test_batch_every_autotune_shape_bit_identical(Q, qhi):
    """Every launch shape the autotuner chooses among -- pipelined, streaming,
    TMEM-staged DEQUE, and shared-memory DEQUE with 1..8 warps per CTA, 8 or
    16 deque entries and one or two scenarios per lane -- gives the same bits
    (tours of 1..500 customers, S = 165: a ragged last tile, and with two
    scenarios per lane a last pair holding one tile)."""
    B, S = 23, 165
    n, tours, coords, dem = _batch(300 + Q, B, S, Q, 1, 500, qhi)
    dem[2][4, 1] = Q + 1
    plan, keep = _plan(n, tours, coords, dem, Q, S)
    ref, refm = plan.run()
    torch.cuda.synchronize()
    ref, refm = ref.clone(), refm.clone()
    shapes = [(-2, 16, 1), (-1, 16, 1), (0, 16, 1)]
    shapes += [(w, r, ns) for w in (1, 2, 4, 8) for r in (8, 16) for ns in (1, 2)]
    tried, tried_ns2 = 0, 0
    for w, r, ns in shapes:
        try:
            info = plan.configure(w, r, ns)
        except api().SdpError as e:
            assert e.code == -5
            continue
        assert (info["warps_per_cta"], info["ring"], info["scenarios_per_lane"]) == (w, r, ns)
        costs, means = plan.run()
        torch.cuda.synchronize()
        assert torch.equal(costs, ref), (w, r, ns)
        assert torch.equal(means.isinf(), refm.isinf())
        tried += 1
        tried_ns2 += ns == 2
    # (uint16 rows of up to 500 customers leave fewer shapes fitting an SM)
    assert tried >= 9 and tried_ns2 >= 2
    assert api().status() & api().FLAG_INFEASIBLE
    plan.close()


@pytest.mark.parametrize("Q,qhi,lengths", [
    (150, 40, [337, 340, 341, 344, 85, 84, 2, 1]),    # uint8 rows: 85 words at n = 340
    (600, 90, [169, 170, 171, 172, 43, 42, 2, 1]),    # uint16 rows: 85 words at n = 170
    (150, 40, [128, 127, 100, 64, 33, 32, 17, 5]),    # every tour n <= 128: six 16 KB stages
])
def test_batch_pipe_narrowing_boundaries(Q, qhi, lengths):
    """Tours on both sides of the narrowing's switch from row groups over all
    its threads (rows of at most 85 words) to one thread per word position,
    and a plan of short tours only (six producer stages): the pipelined
    plan's costs are the per-tour PLAIN kernel's bits, its means the same to
    1e-12, with a ragged last tile (S = 164) and one demand above Q."""
    S = 164
    rng = np.random.default_rng(Q + len(lengths) + lengths[0])
    n = np.array(lengths, np.int32)
    tours = [(rng.permutation(k) + 1).astype(np.int32) for k in n]
    coords = [np.concatenate([[[50, 50]], rng.uniform(0, 100, (k, 2))]).astype(np.float32)
              for k in n]
    dem = [rng.integers(1, qhi + 1, size=(S, k)).astype(np.int32) for k in n]
    dem[1][S - 1, n[1] // 2] = Q + 1
    plan, _ = _plan(n, tours, coords, dem, Q, S)
    plan.configure(-2, 16, 1)
    assert plan.info()["warps_per_cta"] == -2
    api().status()
    costs, means = plan.run()
    torch.cuda.synchronize()
    for b in range(len(n)):
        p = api().split_eval(torch.from_numpy(tours[b]).cuda(), Q,
                             torch.from_numpy(dem[b]).cuda(),
                             coords=torch.from_numpy(coords[b]).cuda(), algo="plain")
        torch.cuda.synchronize()
        assert torch.equal(costs[b], p["cost"]), b
        m, pm = float(means[b]), float(p["mean"])
        assert (np.isinf(m) and np.isinf(pm)) or abs(m - pm) <= 1e-12 * abs(pm), b
    st = api().status()
    assert np.isinf(float(means[1])) and st & api().FLAG_INFEASIBLE
    assert st & api().FLAG_DEVICE_CHECK == 0
    plan.close()


def test_batch_infeasible_and_fallback():
    """Scenarios with a demand above Q and with zero-cost ties (deque ring
    overflow -> plain fallback) inside a batch."""
    B, S, Q = 5, 70, 12
    rng = np.random.default_rng(3)
    n = np.array([40, 7, 33, 1, 20], np.int32)
    tours = [(rng.permutation(k) + 1).astype(np.int32) for k in n]
    coords = [np.full((k + 1, 2), 50.0, np.float32) if b % 2 == 0 else
              np.concatenate([[[50, 50]], rng.uniform(0, 100, (k, 2))]).astype(np.float32)
              for b, k in enumerate(n)]
    dem = [rng.integers(0, 3, size=(S, k)).astype(np.int32) for k in n]
    dem[1][5, 3] = Q + 1
    plan, keep = _plan(n, tours, coords, dem, Q, S)
    costs, means = plan.run()
    torch.cuda.synchronize()
    for b in range(B):
        o = oracle.split(tours[b], Q, dem[b], coords=coords[b])
        g = costs[b].cpu().double().numpy()
        assert np.array_equal(np.isinf(g), np.isinf(o["cost"]))
        f = np.isfinite(g)
        assert np.all(np.abs(g[f] - o["cost"][f]) <= 1e-5 * np.maximum(o["cost"][f], 1e-30))
    assert np.isinf(float(means[1]))
    fl = api().status()
    assert fl & api().FLAG_INFEASIBLE and fl & api().FLAG_FALLBACK
    plan.close()


def test_batch_c4_full_size_sampled():
    """4096 tours, n_b ~ U{20..1000}, S=4096 each (34 GB of demands generated
    on the device), sampled (tour, scenario) pairs checked against the
    oracle and every per-tour mean against the FP32 costs."""
    spec = wl.BATCH_C4
    nb = wl.batch_sizes(spec)
    tours, coords = zip(*(wl.batch_tour(spec, b, int(nb[b])) for b in range(spec.B)))
    dem_off = np.zeros(spec.B, np.int64)
    dem_off[1:] = np.cumsum(nb[:-1].astype(np.int64) * spec.S)
    total = int(dem_off[-1] + nb[-1] * spec.S)
    d = torch.empty(total, dtype=torch.int32, device="cuda")
    for b in range(spec.B):
        seg = d[dem_off[b]:dem_off[b] + nb[b] * spec.S].view(spec.S, int(nb[b]))
        wl.batch_demands_device(spec, b, int(nb[b]), seg)
    t = torch.from_numpy(np.concatenate(tours)).cuda()
    c = torch.from_numpy(np.concatenate(coords)).cuda()
    plan = api().SplitPlan(nb, t, c, d, spec.Q, spec.S, dem_off=dem_off)
    costs, means = plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    for b in rng.choice(spec.B, 48, replace=False):
        rows = np.sort(rng.choice(spec.S, 8, replace=False))
        q = np.concatenate([wl.batch_demands(spec, int(b), int(nb[b]), int(s), int(s) + 1)
                            for s in rows])
        np.testing.assert_array_equal(
            q, d[dem_off[b]:dem_off[b] + nb[b] * spec.S].view(spec.S, -1)[rows].cpu().numpy())
        o = oracle.split(tours[b], spec.Q, q, coords=coords[b])
        g = costs[int(b)][rows].cpu().double().numpy()
        assert (np.abs(g - o["cost"]) / o["cost"]).max() <= 1e-5
    host_means = costs.double().mean(1)
    assert torch.allclose(means, host_means, rtol=1e-12, atol=0)
    assert api().status() & (api().FLAG_INFEASIBLE | api().FLAG_FALLBACK) == 0
    plan.close()

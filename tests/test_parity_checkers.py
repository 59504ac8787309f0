"""The GPU parity checks themselves (tests/gpu_util.py), on CPU: fed the
oracle's own results in the GPU's output types they pass; fed the same
results with one mistake planted -- a cost off by more than the tolerance,
infeasibility flipped, a predecessor or policy changed where the optimum is
unique, a missing sentinel -- they fail, so a parity test cannot pass by
comparing nothing.  Changes at near-ties pass, as the tolerance states."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_util import MARGIN, check_reinsert, check_split, preds_to_i64


def _split_case():
    rng = np.random.default_rng(31)
    n, S, Q = 30, 60, 40
    xy = np.empty((n + 1, 2), np.float32)
    xy[0] = (50, 50)
    xy[1:] = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    tour = (rng.permutation(n) + 1).astype(np.int32)
    q = rng.integers(1, 15, size=(S, n)).astype(np.int32)
    q[7, 3] = Q + 1                       # one infeasible scenario
    orc = oracle.split(tour, Q, q, coords=xy, want_margin=True)
    return orc


def _gpu_like(orc, u16=False):
    cost = torch.from_numpy(orc["cost"].astype(np.float32))
    p = orc["pred"].astype(np.int32)
    pred = torch.from_numpy(p.astype(np.uint16).view(np.int16) if u16 else p)
    return cost, pred


@pytest.mark.parametrize("u16", [False, True])
def test_check_split_passes_the_oracles_own_results(u16):
    orc = _split_case()
    cost, pred = _gpu_like(orc, u16)
    assert check_split(cost, pred, orc) >= 0.5
    check_split(cost, None, orc)


def test_check_split_catches_each_planted_mistake():
    orc = _split_case()
    unique = np.argwhere((orc["pred"] >= 0) & (orc["margin"] > MARGIN))
    near = np.argwhere((orc["pred"] >= 1) & (orc["margin"] <= MARGIN))
    s, i = unique[len(unique) // 2]

    cost, pred = _gpu_like(orc)
    cost[0] = float(orc["cost"][0] * (1 + 3e-5))
    with pytest.raises(AssertionError, match="rel err"):
        check_split(cost, pred, orc)

    cost, pred = _gpu_like(orc)
    cost[7] = 1.0                         # the infeasible scenario reported finite
    with pytest.raises(AssertionError, match="infeasibility"):
        check_split(cost, pred, orc)

    cost, pred = _gpu_like(orc)
    pred[s, i] = int(pred[s, i]) - 1 if int(pred[s, i]) > 0 else int(pred[s, i]) + 1
    with pytest.raises(AssertionError, match="predecessor mismatches"):
        check_split(cost, pred, orc)

    cost, pred = _gpu_like(orc)
    pred[7, -1] = 0                       # a sentinel (-1) replaced by a position
    with pytest.raises(AssertionError):
        check_split(cost, pred, orc)

    # a change at a near-tie passes (if the case has one), and a case where
    # too few positions are unique enough to check is refused
    if len(near):
        cost, pred = _gpu_like(orc)
        ns, ni = near[0]
        pred[ns, ni] = int(pred[ns, ni]) - 1
        check_split(cost, pred, orc)
    cost, pred = _gpu_like(orc)
    flat = dict(orc, margin=np.zeros_like(orc["margin"]))
    with pytest.raises(AssertionError, match="unique enough"):
        check_split(cost, pred, flat)
    check_split(cost, pred, flat, min_checked=0.0)


def test_preds_to_i64_reads_uint16_bits():
    p = torch.from_numpy(np.array([[0, 1, 40000, 65534, 65535]], np.uint16).view(np.int16))
    assert preds_to_i64(p).tolist() == [[0, 1, 40000, 65534, -1]]
    assert preds_to_i64(torch.tensor([[3, -1]], dtype=torch.int32)).tolist() == [[3, -1]]


def _reinsert_case():
    rng = np.random.default_rng(32)
    T, U, S, I0 = 12, 20, 40, 10
    fixed = rng.uniform(5, 50, T).astype(np.float32)
    cons = rng.poisson(4, size=(S, T)).astype(np.int32)
    orc = oracle.reinsert(T, U, I0, 1.0, 20.0, 0.0, fixed, cons, want_margin=True)
    return orc, cons, U, I0


def test_check_reinsert_passes_and_catches_planted_mistakes():
    orc, cons, U, I0 = _reinsert_case()
    val = torch.from_numpy(orc["value"].astype(np.float32))
    pol = torch.from_numpy(orc["policy"].copy())
    checked = check_reinsert(val, pol, orc, cons, U, I0)
    assert checked >= 0.9 * pol.numel()

    bad = val.clone()
    bad[3] = float(orc["value"][3] * (1 + 3e-5))
    with pytest.raises(AssertionError, match="rel err"):
        check_reinsert(bad, pol, orc, cons, U, I0)

    # flip the first day's decision of a scenario where it is clear
    s = next(s for s in range(pol.shape[0]) if orc["margin"][s, 0, I0] > MARGIN)
    flipped = pol.clone()
    flipped[s, 0] = 1 - int(flipped[s, 0])
    with pytest.raises(AssertionError):
        check_reinsert(val, flipped, orc, cons, U, I0)

    # at a near-tie the paths may part: the comparison of that scenario stops
    tied = dict(orc, margin=orc["margin"].copy())
    tied["margin"][s, 0, I0] = 0.0
    fewer = check_reinsert(val, flipped, tied, cons, U, I0)
    assert fewer < checked

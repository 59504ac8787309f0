"""Shared checks for the GPU parity tests (CUDA path vs the FP64 oracle).

Tolerances (stated by the build's precision contract): costs and values
within 1e-5 relative of the FP64 oracle; predecessors and policies bit-exact
wherever the oracle's optimum is unique by more than 1e-4 relative (the
oracle reports the relative gap between the best and second-best candidate).
"""
import numpy as np

RTOL = 1e-5
MARGIN = 1e-4


def preds_to_i64(p):
    a = p.cpu().numpy()
    if a.dtype == np.int16:
        a = a.astype(np.int64) & 0xFFFF
        a[a == 0xFFFF] = -1
    return a.astype(np.int64)


def check_split(cost, pred, orc, rows=None, rtol=RTOL, margin=MARGIN, min_checked=0.5):
    """cost fp32 [S'] (torch), pred [S', n] or None; orc = oracle.split(...)
    dict over the same scenarios (rows selects GPU rows if given)."""
    c = cost.detach().cpu().double().numpy()
    if rows is not None:
        c = c[rows]
    oc = orc["cost"]
    assert c.shape == oc.shape
    assert np.array_equal(np.isinf(c), np.isinf(oc)), "infeasibility differs"
    fin = np.isfinite(oc)
    if fin.any():
        rel = np.abs(c[fin] - oc[fin]) / np.maximum(np.abs(oc[fin]), 1e-300)
        assert rel.max() <= rtol, f"max rel err {rel.max():.3e}"
    if pred is None:
        return
    gp = preds_to_i64(pred)
    if rows is not None:
        gp = gp[rows]
    op = orc["pred"].astype(np.int64)
    assert gp.shape == op.shape
    # where the oracle's J(i) is +inf the GPU writes the sentinel
    assert np.array_equal(gp[op == -1], op[op == -1])
    mask = (op >= 0) & (orc["margin"] > margin)
    bad = np.argwhere(gp[mask] != op[mask])
    assert bad.size == 0, f"{bad.size} predecessor mismatches"
    frac = mask.sum() / max(1, (op >= 0).sum())
    assert frac >= min_checked, f"only {frac:.2%} of predecessors are unique enough to check"
    return frac


def check_reinsert(value, policy, orc, cons, U, I0, rows=None, rtol=RTOL, margin=MARGIN):
    """value fp32 [S'], policy uint8 [S', T] (torch); orc = oracle.reinsert(...,
    want_margin=True) over the same scenarios; cons int32 [S, T] numpy.
    Policies are compared along the oracle's optimal path: bit-exact at every
    day whose decision is unique by more than `margin`; at a near-tie the
    paths may part, and the comparison of that scenario stops there."""
    v = value.detach().cpu().double().numpy()
    if rows is not None:
        v = v[rows]
    ov = orc["value"]
    rel = np.abs(v - ov) / np.maximum(np.abs(ov), 1e-300)
    ok = (rel <= rtol) | (np.abs(v - ov) <= 1e-6)
    assert ok.all(), f"max rel err {rel.max():.3e}"
    if policy is None:
        return
    gp = policy.cpu().numpy()
    if rows is not None:
        gp = gp[rows]
    op = orc["policy"]
    mg = orc["margin"]
    S, T = op.shape
    checked = 0
    for s in range(S):
        I = I0
        for t in range(T):
            if mg[s, t, I] > margin:
                assert gp[s, t] == op[s, t], (s, t, I)
                checked += 1
            elif gp[s, t] != op[s, t]:
                break
            q = (U - I) if op[s, t] else 0
            I = max(0, I + q - int(cons[s, t]))
    return checked

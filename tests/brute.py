"""Brute-force enumerators used to pin the oracle (pure Python, tiny sizes).

They share nothing with the oracle's code: Split is solved by listing every
set of cut points of the giant tour, reinsertion by simulating every one of
the 2^T delivery sequences forward in time.
"""
import itertools
import math


def euclid(coords, a, b):
    dx = float(coords[a][0]) - float(coords[b][0])
    dy = float(coords[a][1]) - float(coords[b][1])
    return math.sqrt(dx * dx + dy * dy)


def split_brute(tour, q_by_customer, Q, cost, max_routes=None):
    """Min over all partitions of the tour into consecutive routes whose load
    is <= Q (and, if max_routes is given, into at most that many routes) of
    the summed route costs (depot -> customers in tour order -> depot).
    cost(a, b) gives the travel cost between nodes (0 = depot).  Returns
    (best cost, list of optimal partitions as lists of routes)."""
    n = len(tour)
    if n == 0:
        return 0.0, [[]]
    best, arg = math.inf, []
    for mask in range(1 << (n - 1)):
        cuts = [k for k in range(1, n) if mask >> (k - 1) & 1]
        if max_routes is not None and len(cuts) + 1 > max_routes:
            continue
        bounds = [0] + cuts + [n]
        total, ok = 0.0, True
        routes = []
        for a, b in zip(bounds[:-1], bounds[1:]):
            seg = tour[a:b]
            if sum(q_by_customer[c - 1] for c in seg) > Q:
                ok = False
                break
            r = cost(0, seg[0]) + cost(seg[-1], 0)
            for x, y in zip(seg[:-1], seg[1:]):
                r += cost(x, y)
            total += r
            routes.append(list(seg))
        if not ok:
            continue
        tol = 1e-12 * max(1.0, abs(total))
        if best == math.inf or total < best - tol:
            best, arg = total, [routes]
        elif abs(total - best) <= tol:
            arg.append(routes)
    return best, arg


def split_soft_brute(tour, q_by_customer, Q, beta, cost):
    """Min over ALL partitions of the tour into consecutive routes of the
    summed route costs plus beta per unit of each route's load above Q.
    Returns (best cost, list of optimal partitions)."""
    n = len(tour)
    if n == 0:
        return 0.0, [[]]
    best, arg = math.inf, []
    for mask in range(1 << (n - 1)):
        cuts = [k for k in range(1, n) if mask >> (k - 1) & 1]
        bounds = [0] + cuts + [n]
        total = 0.0
        routes = []
        for a, b in zip(bounds[:-1], bounds[1:]):
            seg = tour[a:b]
            load = sum(q_by_customer[c - 1] for c in seg)
            r = cost(0, seg[0]) + cost(seg[-1], 0)
            for x, y in zip(seg[:-1], seg[1:]):
                r += cost(x, y)
            total += r + beta * max(0, load - Q)
            routes.append(list(seg))
        tol = 1e-12 * max(1.0, abs(total))
        if best == math.inf or total < best - tol:
            best, arg = total, [routes]
        elif abs(total - best) <= tol:
            arg.append(routes)
    return best, arg


def reinsert_brute(T, U, I0, h, p, unit_cost, fixed, cons, H=None):
    """Min over all 2^T delivery sequences of the simulated total cost.
    Returns (best value, list of optimal 0/1 sequences)."""
    best, arg = math.inf, []
    for seq in itertools.product((0, 1), repeat=T):
        I, total = I0, 0.0
        for t, a in enumerate(seq):
            q = (U - I) if a else 0
            if q > 0:
                total += float(fixed[t]) + unit_cost * q
            x = I + q - int(cons[t])
            if H is not None:
                total += H[max(0, x)]
            else:
                total += h * x if x >= 0 else p * (-x)
            I = max(0, x)
        tol = 1e-12 * max(1.0, abs(total))
        if best == math.inf or total < best - tol:
            best, arg = total, [seq]
        elif abs(total - best) <= tol:
            arg.append(seq)
    return best, arg


def reinsert_routes_brute(T, U, I0, h, p, unit_cost, rcost, cap, cons, H=None):
    """Min over every sequence of daily actions (0 = no delivery, r + 1 =
    deliver up to U on route r, allowed when cap[t][r] >= U - I) of the
    simulated total cost.  Returns (best value, list of optimal sequences)."""
    K = len(rcost[0]) if T else 0
    best, arg = math.inf, []
    for seq in itertools.product(range(K + 1), repeat=T):
        I, total, ok = I0, 0.0, True
        for t, a in enumerate(seq):
            q = (U - I) if a else 0
            if a:
                if q == 0 or cap[t][a - 1] < q:
                    ok = False
                    break
                total += float(rcost[t][a - 1]) + unit_cost * q
            x = I + q - int(cons[t])
            if H is not None:
                total += H[max(0, x)]
            else:
                total += h * x if x >= 0 else p * (-x)
            I = max(0, x)
        if not ok:
            continue
        tol = 1e-12 * max(1.0, abs(total))
        if best == math.inf or total < best - tol:
            best, arg = total, [seq]
        elif abs(total - best) <= tol:
            arg.append(seq)
    return best, arg


def _day_cost(t, I, a, U, h, p, unit_cost, fixed_or_rcost, cons, H, routes):
    """Cost of action a on day t from start-of-day inventory I and the next
    state; None when the action is not allowed.  a = 0: no delivery; a = 1
    (two-action DP) or r + 1 (route r): refill to U."""
    q = (U - I) if a else 0
    day = 0.0
    if a:
        if routes:
            rcost, cap = fixed_or_rcost
            if q == 0 or cap[t][a - 1] < q:
                return None
            day += float(rcost[t][a - 1]) + unit_cost * q
        elif q > 0:
            day += float(fixed_or_rcost[t]) + unit_cost * q
    x = I + q - int(cons[t])
    if H is not None:
        day += H[max(0, x)]
    else:
        day += h * x if x >= 0 else p * (-x)
    return day, max(0, x)


def reinsert_action_values(T, U, h, p, unit_cost, fixed, cons, t, I, H=None, rcost=None,
                           cap=None):
    """Value of each allowed action at (day t, start-of-day inventory I) when
    every later day acts optimally, by simulating every continuation sequence.
    Two-action DP (fixed given): actions 0 and 1 (1 only if I < U).  Route
    options (rcost [T][K], cap [T][K] given): 0 and r + 1 for every route
    whose capacity holds U - I.  Returns {action: value}."""
    routes = rcost is not None
    par = (rcost, cap) if routes else fixed
    K = len(rcost[0]) if routes else 1
    first = [0] + ([a for a in range(1, K + 1)] if I < U else [])
    out = {}
    for a0 in first:
        r0 = _day_cost(t, I, a0, U, h, p, unit_cost, par, cons, H, routes)
        if r0 is None:
            continue
        best = math.inf
        for seq in itertools.product(range(K + 1), repeat=T - t - 1):
            total, J, ok = r0[0], r0[1], True
            for k, a in enumerate(seq):
                r = _day_cost(t + 1 + k, J, a, U, h, p, unit_cost, par, cons, H, routes)
                if r is None or (a and J == U):
                    ok = False
                    break
                total += r[0]
                J = r[1]
            if ok:
                best = min(best, total)
        out[a0] = best
    return out


def split_candidates(tour, q_by_customer, Q, cost, i, beta=None):
    """Every candidate value of J(i) in Eq. eqdpA: for each predecessor p < i,
    the brute-force optimum over the first p customers plus the cost of the
    route s_{p+1..i}.  Hard capacity (beta None): only routes of load <= Q;
    soft capacity: every route, plus beta per unit of load above Q.
    Returns a list of (value, p)."""
    out = []
    for p in range(i):
        seg = tour[p:i]
        load = sum(q_by_customer[c - 1] for c in seg)
        if beta is None and load > Q:
            continue
        if beta is None:
            prev = split_brute(tour[:p], q_by_customer, Q, cost)[0]
        else:
            prev = split_soft_brute(tour[:p], q_by_customer, Q, beta, cost)[0]
        if prev == math.inf:
            continue
        r = cost(0, seg[0]) + cost(seg[-1], 0)
        for x, y in zip(seg[:-1], seg[1:]):
            r += cost(x, y)
        if beta is not None:
            r += beta * max(0, load - Q)
        out.append((prev + r, p))
    return out

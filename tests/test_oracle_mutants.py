"""The oracle's pins catch plausible mistakes.  Each mutant below is a copy of
oracle/sdp_oracle.c with one mistake planted in it -- a dropped term, a wrong
sign, an index off by one, a transposed operand, a tie rule or a margin
taken the other way -- compiled on the CPU into a library of its own.  The
pin files (tests/test_oracle_*.py) then run, in a child process, against
that library instead of the real one, and at least one pin must fail.  A
control copy with no mistake must pass them all.  No mutant reads or writes
outside its arrays, so each one only computes a wrong answer."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "sdp_oracle.c")
PIN_FILES = ["tests/test_oracle_split.py", "tests/test_oracle_split_soft.py",
             "tests/test_oracle_split_fleet.py", "tests/test_oracle_reinsert.py",
             "tests/test_oracle_reinsert_routes.py", "tests/test_oracle_saa.py"]

# (name, text in the oracle, replacement, which occurrence of the text)
MUTANTS = [
    # Split (Eq. eqdpA): route cost W, capacity window, arcs, ties, margin
    ("split: return leg dropped", "const double W = cost_ab(c, 0, sp1) + inner + back;",
     "const double W = cost_ab(c, 0, sp1) + inner;", 0),
    ("split: capacity off by one", "if (load > Q) break;", "if (load >= Q) break;", 0),
    ("split: inner arc transposed", "inner += cost_ab(c, sp1, tour[p + 1]);",
     "inner += cost_ab(c, tour[p + 1], sp1);", 0),
    ("split: ties to the largest p", "if (cand <= best)", "if (cand < best)", 0),
    ("split: margin over the second best",
     "margin[i - 1] = (second - best) / fmax(fabs(best), 1e-300);",
     "margin[i - 1] = (second - best) / fmax(fabs(second), 1e-300);", 0),
    ("split: infinite J(p) not skipped", "if (isinf(J[p])) continue;", "", 0),
    # soft capacity: the penalty term, its threshold, ties
    ("soft: penalty sign", "const double cand = J[p] + W + beta * excess;",
     "const double cand = J[p] + W - beta * excess;", 0),
    ("soft: excess off by one", "load > Q ? (double)(load - Q) : 0.0",
     "load >= Q ? (double)(load - Q + 1) : 0.0", 0),
    ("soft: ties to the largest p", "if (cand <= best)", "if (cand < best)", 2),
    # fleet-limited Split: the layer below, ties over route counts, labels
    ("fleet: same layer instead of the one below", "const double prev = J[(k - 1) * w + p];",
     "const double prev = J[k * w + p];", 0),
    ("fleet: ties to the most routes", 'if (v < best) {  /* "<": the fewest routes on ties */',
     "if (v <= best) {", 0),
    ("fleet: route labels shifted", "route[m] = k - 1;", "route[m] = k;", 0),
    ("fleet: capacity off by one", "if (load > Q) break;", "if (load >= Q) break;", 1),
    # explicit matrix A of the Split
    ("matrix: first customer's load dropped",
     "for (int k = p + 1; k <= i; ++k) load += q_by_customer[tour[k - 1] - 1];",
     "for (int k = p + 2; k <= i; ++k) load += q_by_customer[tour[k - 1] - 1];", 0),
    ("min-plus: J subtracted", "double v = a + J[i];", "double v = a - J[i];", 0),
    # gradient and route counts
    ("gradient: depot arc transposed", "grad_out[(size_t)0 * m + tour[p]] += 1.0;",
     "grad_out[(size_t)tour[p] * m + 0] += 1.0;", 0),
    ("gradient: first inner arc dropped", "for (int k = p + 1; k < i; ++k)\n        grad_out",
     "for (int k = p + 2; k < i; ++k)\n        grad_out", 0),
    ("route counts: end taken at the start", "end_cnt[i - 1] += 1;", "end_cnt[p] += 1;", 0),
    # reinsertion (Alg. SolveBatchDP, Eq. eqdp2)
    ("reinsert: route cost dropped",
     "double dv = route_cost(m, t, q) + end_cost(m, x1) + Cn[x1 > 0 ? x1 : 0];",
     "double dv = end_cost(m, x1) + Cn[x1 > 0 ? x1 : 0];", 0),
    ("reinsert: next state not shifted", "double nd = end_cost(m, x0) + Cn[x0 > 0 ? x0 : 0];",
     "double nd = end_cost(m, x0) + Cn[I];", 0),
    ("reinsert: ties deliver", "if (dv < nd) { best = dv; a = 1; }",
     "if (dv <= nd) { best = dv; a = 1; }", 0),
    ("reinsert: backtrack refill one short", "int64_t q = a ? (U - I) : 0;",
     "int64_t q = a ? (U - I - 1) : 0;", 0),
    ("reinsert: lost-sales sign", "m->p * (double)(-x);", "m->p * (double)(x);", 0),
    ("reinsert: margin halved", "mg = den > 0 ? fabs(dv - nd) / den",
     "mg = den > 0 ? fabs(dv - nd) / (2 * den)", 0),
    ("reinsert: unit cost dropped", "m->unit_cost * (double)q : 0.0", "0.0 : 0.0", 0),
    ("forward: end cost dropped", "double c = route_cost(&m, t, q) + end_cost(&m, x);",
     "double c = route_cost(&m, t, q);", 0),
    # route options
    ("routes: capacity test off by one", "if (cap[(size_t)t * K + r] < q) continue;",
     "if (cap[(size_t)t * K + r] <= q) continue;", 0),
    ("routes: ties to the last route", "if (dv < best) {", "if (dv <= best) {", 0),
    ("routes: policy label", "a = (uint8_t)(r + 1);", "a = (uint8_t)(r + 1 + (r > 0));", 0),
]


def _replace_nth(src, old, new, occ):
    at = -1
    for _ in range(occ + 1):
        at = src.find(old, at + 1)
        assert at >= 0, f"oracle text not found: {old!r} (occurrence {occ})"
    return src[:at] + new + src[at + len(old):]


def run_mutant(m):
    """Compile the oracle with mutant m planted (None: unchanged) and run the
    pin files against it in a child process: (exit code, last output line)."""
    name, old, new, occ = m
    with open(ORACLE_C) as f:
        src = f.read()
    if old is not None:
        src = _replace_nth(src, old, new, occ)
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        c = os.path.join(d, "sdp_oracle.c")
        with open(c, "w") as f:
            f.write(src)
        lib = os.path.join(d, "liboracle.so")
        script = ("import sys, pytest, oracle\n"
                  f"oracle._SRC = {c!r}\noracle._LIB_PATH = {lib!r}\noracle._lib = None\n"
                  "sys.exit(pytest.main(['-x', '-q', '-m', 'not gpu', '-p', 'no:cacheprovider', "
                  f"'-W', 'ignore', *{PIN_FILES!r}]))\n")
        env = dict(os.environ, OMP_NUM_THREADS="2")
        p = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=900)
        lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
        return p.returncode, (lines[-1] if lines else p.stderr[-300:])
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_every_planted_mistake_fails_a_pin():
    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(run_mutant, MUTANTS))
    survived = [(m[0], tail) for m, (rc, tail) in zip(MUTANTS, res) if rc == 0]
    broken = [(m[0], rc, tail) for m, (rc, tail) in zip(MUTANTS, res) if rc not in (0, 1)]
    assert not broken, broken   # 1 = a pin failed; anything else is a harness error
    assert not survived, survived


def test_unplanted_copy_passes_every_pin():
    rc, tail = run_mutant(("control", None, None, 0))
    assert rc == 0, tail

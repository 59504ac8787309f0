"""The oracle's pins catch plausible mistakes.  Each mutant below is a copy of
oracle/sdp_oracle.c (compiled on the CPU into a library of its own) or of
oracle/saa.py (executed into the imported module) with one mistake planted
in it -- a dropped term, a wrong sign, an index off by one, a transposed
operand, a tie rule or a margin taken the other way.  The pin files
(tests/test_oracle_*.py) then run, in a child process, against that copy
instead of the real one, and at least one pin must fail.  A control copy
with no mistake must pass them all.  No mutant reads or writes outside its
arrays, so each one only computes a wrong answer."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "sdp_oracle.c")
ORACLE_SAA = os.path.join(ROOT, "oracle", "saa.py")
PIN_FILES = ["tests/test_oracle_split.py", "tests/test_oracle_split_soft.py",
             "tests/test_oracle_split_fleet.py", "tests/test_oracle_reinsert.py",
             "tests/test_oracle_reinsert_routes.py", "tests/test_oracle_saa.py"]

# (name, text in oracle/sdp_oracle.c, replacement, which occurrence of the text)
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
    ("routes: margin halved", "(den > 0 ? (second - best) / den : 0.0)",
     "(den > 0 ? (second - best) / (2 * den) : 0.0)", 0),
    ("routes: end state from I", "const int64_t x1 = (int64_t)U - dt;",
     "const int64_t x1 = (int64_t)I - dt;", 0),
    ("routes: backtrack state", "const int64_t x = (a ? U : I) - d[t];",
     "const int64_t x = (a ? U - 1 : I) - d[t];", 0),
    # the sample means, the fleet margin along the path, the last layer
    ("split: mean over S - 1", "*mean_out = S > 0 ? sum / (double)S : 0.0;",
     "*mean_out = S > 1 ? sum / (double)(S - 1) : 0.0;", 0),
    ("fleet: mean over S - 1", "*mean_out = S > 0 ? sum / (double)S : 0.0;",
     "*mean_out = S > 1 ? sum / (double)(S - 1) : 0.0;", 1),
    ("soft: mean over S - 1", "*mean_out = S > 0 ? sum / (double)S : 0.0;",
     "*mean_out = S > 1 ? sum / (double)(S - 1) : 0.0;", 2),
    ("reinsert: mean over S - 1", "*mean_out = S > 0 ? sum / (double)S : 0.0;",
     "*mean_out = S > 1 ? sum / (double)(S - 1) : 0.0;", 3),
    ("fleet: path margin ignored", "mg = fmin(mg, M[k * w + i]);", "mg = mg;", 0),
    ("fleet: last layer ignored", "for (int k = 1; k <= K; ++k) {\n    const double v",
     "for (int k = 1; k < K; ++k) {\n    const double v", 0),
    # the forward recursion, the terminal and table costs, the C_0 table, arcs
    ("forward: last action overwrites", "if (c < *a) *a = c;", "*a = c;", 0),
    ("reinsert: value0 of day 1", "for (int I = 0; I < W; ++I) value0[I] = C[I];",
     "for (int I = 0; I < W; ++I) value0[I] = C[(T > 1 ? W : 0) + I];", 0),
    ("reinsert: terminal cost 1", "for (int I = 0; I < W; ++I) C[(size_t)T * W + I] = 0.0;",
     "for (int I = 0; I < W; ++I) C[(size_t)T * W + I] = 1.0;", 0),
    ("reinsert: table end cost shifted",
     "if (m->H) return m->H[x > 0 ? (x > m->U ? m->U : x) : 0];",
     "if (m->H) return m->H[x > 1 ? (x > m->U ? m->U : x - 1) : 0];", 0),
    ("split: arcs miss p = 0",
     "++narcs;\n      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);\n      if (isinf",
     "narcs += p > 0;\n      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);\n      if (isinf",
     0),
    ("soft: arcs miss p = 0",
     "      ++narcs;\n      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);\n      const double W",
     "      narcs += p > 0;\n      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);\n"
     "      const double W", 0),
    # single-candidate margins, the explicit matrix's last predecessor, distances
    ("matrix: last predecessor left out",
     "for (int p = 0; p < i; ++p) col[p] = A_out[(size_t)p * m + i];",
     "for (int p = 0; p < i; ++p) col[p] = p == i - 1 ? INFINITY : A_out[(size_t)p * m + i];", 0),
    ("split: single-candidate margin 0",
     "if (bestp < 0 || isinf(second)) margin[i - 1] = INFINITY;",
     "if (bestp < 0 || isinf(second)) margin[i - 1] = 0.0;", 0),
    ("soft: single-candidate margin 0",
     "if (bestp < 0 || isinf(second)) margin[i - 1] = INFINITY;",
     "if (bestp < 0 || isinf(second)) margin[i - 1] = 0.0;", 1),
    ("reinsert: margin at I = U is 0", "double mg = INFINITY;", "double mg = 0.0;", 1),
    ("euclid: squared distance", "return sqrt(dx * dx + dy * dy);", "return dx * dx + dy * dy;", 0),
    # fleet routes and margin, gradient scale, route counts, value0, route backtrack
    ("fleet: first customer of a route unlabelled", "for (int m = p; m < i; ++m) route[m] = k - 1;",
     "for (int m = p + 1; m < i; ++m) route[m] = k - 1;", 0),
    ("fleet: margin of the layer choice ignored",
     "double mg = (bestk == 0 || isinf(second)) ? INFINITY : (second - best) / fmax(fabs(best), 1e-300);",
     "double mg = INFINITY;", 0),
    ("gradient: over S + 1",
     "for (size_t e = 0; e < (size_t)m * m; ++e) grad_out[e] /= (double)S;",
     "for (size_t e = 0; e < (size_t)m * m; ++e) grad_out[e] /= (double)(S + 1);", 0),
    ("route counts: skipped not counted", "if (!ok) { ++skip; continue; }",
     "if (!ok) { continue; }", 0),
    ("reinsert: value0 skipped for I = U", "for (int I = 0; I < W; ++I) value0[I] = C[I];",
     "for (int I = 0; I < W - 1; ++I) value0[I] = C[I];", 0),
    ("routes: backtrack refills on route 1 only", "const int64_t x = (a ? U : I) - d[t];",
     "const int64_t x = (a > 1 ? U : I) - d[t];", 0),
]

# the same for oracle/saa.py (the SAA search: SplitMix64, moves, selection)
SAA_MUTANTS = [
    ("saa: counter off by one", "z = (seed + (c + 1) * GAMMA) & M64",
     "z = (seed + c * GAMMA) & M64", 0),
    ("saa: finaliser shift", "z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64",
     "z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & M64", 0),
    ("saa: position a from the high word", "a = (z & 0xFFFFFFFF) % n", "a = (z >> 32) % n", 0),
    ("saa: b skips a strictly", "if b >= a:\n        b += 1", "if b > a:\n        b += 1", 0),
    ("saa: kind from the wrong byte", "((z >> 32) & 0xFF)", "((z >> 33) & 0xFF)", 0),
    ("saa: 2-opt one short", "t[a:b + 1] = t[a:b + 1][::-1]", "t[a:b] = t[a:b][::-1]", 0),
    ("saa: relocate one further", "t.insert(b, x)", "t.insert(b + 1, x)", 0),
    ("saa: equal score accepted", "take = ms[kbest] < m0", "take = ms[kbest] <= m0", 0),
    ("saa: last minimum taken", "kbest = int(np.argmin(ms))",
     "kbest = len(ms) - 1 - int(np.argmin(ms[::-1]))", 0),
    ("saa: trace of a rejected step", "trace.append(ms[kbest] if take else m0)",
     "trace.append(ms[kbest])", 0),
]


def _replace_nth(src, old, new, occ):
    at = -1
    for _ in range(occ + 1):
        at = src.find(old, at + 1)
        assert at >= 0, f"oracle text not found: {old!r} (occurrence {occ})"
    return src[:at] + new + src[at + len(old):]


def run_mutant(m, target=ORACLE_C):
    """Plant mutant m (None: no change) in a copy of target -- the C oracle,
    compiled into a library of its own, or the SAA oracle, executed into the
    imported module -- and run the pin files against it in a child process:
    (exit code, last output line)."""
    name, old, new, occ = m
    with open(target) as f:
        src = f.read()
    if old is not None:
        src = _replace_nth(src, old, new, occ)
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        c = os.path.join(d, os.path.basename(target))
        with open(c, "w") as f:
            f.write(src)
        script = "import sys, pytest, oracle, oracle.saa\n"
        if target == ORACLE_C:
            lib = os.path.join(d, "liboracle.so")
            script += (f"oracle._SRC = {c!r}\noracle._LIB_PATH = {lib!r}\n"
                       "oracle._lib = None\n")
        else:
            # the package re-exports the search's functions: rebind those too
            script += (f"exec(compile(open({c!r}).read(), oracle.saa.__file__, 'exec'), "
                       "oracle.saa.__dict__)\n"
                       "for k in ('apply_move', 'draw_move', 'saa_search', 'splitmix64'):\n"
                       "    setattr(oracle, k, getattr(oracle.saa, k))\n")
        script += ("sys.exit(pytest.main(['-x', '-q', '-m', 'not gpu', '-p', 'no:cacheprovider', "
                   f"'-W', 'ignore', *{PIN_FILES!r}]))\n")
        env = dict(os.environ, OMP_NUM_THREADS="2")
        p = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=900)
        lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
        return p.returncode, (lines[-1] if lines else p.stderr[-300:])
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_every_planted_mistake_fails_a_pin():
    jobs = [(m, ORACLE_C) for m in MUTANTS] + [(m, ORACLE_SAA) for m in SAA_MUTANTS]
    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda j: run_mutant(*j), jobs))
    survived = [(j[0][0], tail) for j, (rc, tail) in zip(jobs, res) if rc == 0]
    broken = [(j[0][0], rc, tail) for j, (rc, tail) in zip(jobs, res) if rc not in (0, 1)]
    assert not broken, broken   # 1 = a pin failed; anything else is a harness error
    assert not survived, survived


@pytest.mark.parametrize("target", [ORACLE_C, ORACLE_SAA])
def test_unplanted_copy_passes_every_pin(target):
    rc, tail = run_mutant(("control", None, None, 0), target)
    assert rc == 0, tail


def test_oracle_has_no_undefined_behaviour_on_the_pins(tmp_path):
    """The C oracle built with UndefinedBehaviorSanitizer, stopping at the
    first finding (signed overflow, shifts out of range, array indexes out of
    bounds, misaligned loads), passes every pin."""
    src = tmp_path / "sdp_oracle.c"
    shutil.copy(ORACLE_C, src)
    lib = tmp_path / "liboracle.so"
    cc = subprocess.run(["gcc", "-std=c11", "-O1", "-fopenmp", "-ffp-contract=off",
                         "-fno-fast-math", "-fPIC", "-shared", "-fsanitize=undefined",
                         "-fno-sanitize-recover=all", str(src), "-o", str(lib), "-lm"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        pytest.skip("no UndefinedBehaviorSanitizer runtime: " + cc.stderr[-200:])
    script = ("import os, sys, pytest, oracle\n"
              f"oracle._SRC = {str(src)!r}\noracle._LIB_PATH = {str(lib)!r}\noracle._lib = None\n"
              f"os.utime({str(lib)!r})\n"
              "sys.exit(pytest.main(['-x', '-q', '-m', 'not gpu', '-p', 'no:cacheprovider', "
              f"'-W', 'ignore', *{PIN_FILES!r}]))\n")
    p = subprocess.run([sys.executable, "-c", script], cwd=ROOT, capture_output=True,
                       text=True, timeout=900, env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert p.returncode == 0, (p.stdout[-1500:], p.stderr[-1500:])


def test_oracle_has_no_memory_errors_on_the_pins(tmp_path):
    """The C oracle built with AddressSanitizer (out-of-bounds and
    use-after-free accesses, reported and fatal) passes every pin.  The
    sanitizer's runtime has to be loaded first, so the child Python starts
    with it preloaded."""
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no AddressSanitizer runtime")
    src = tmp_path / "sdp_oracle.c"
    shutil.copy(ORACLE_C, src)
    lib = tmp_path / "liboracle.so"
    cc = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fopenmp", "-ffp-contract=off",
                         "-fno-fast-math", "-fPIC", "-shared", "-fsanitize=address",
                         "-fno-omit-frame-pointer", str(src), "-o", str(lib), "-lm"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        pytest.skip("AddressSanitizer build failed: " + cc.stderr[-200:])
    script = ("import os, sys, pytest, oracle\n"
              f"oracle._SRC = {str(src)!r}\noracle._LIB_PATH = {str(lib)!r}\noracle._lib = None\n"
              f"os.utime({str(lib)!r})\n"
              "sys.exit(pytest.main(['-x', '-q', '-m', 'not gpu', '-p', 'no:cacheprovider', "
              f"'-W', 'ignore', *{PIN_FILES!r}]))\n")
    env = dict(os.environ, OMP_NUM_THREADS="2", LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:verify_asan_link_order=0:abort_on_error=1")
    p = subprocess.run([sys.executable, "-c", script], cwd=ROOT, capture_output=True,
                       text=True, timeout=900, env=env)
    assert p.returncode == 0, (p.stdout[-1500:], p.stderr[-1500:])

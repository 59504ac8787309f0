"""The bench's host-side logic, on CPU: the reference arm's JSON line (the
FP64 oracle timed on bounded samples of the bench workload), its argument
check and rank handling, the clock record's reading of nvidia-smi samples,
the per-result error summaries against the oracle, the arithmetic of the
stored DRAM traffic records, and the hash that tells whether those records
still describe the kernel being timed."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=e, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = _run("--impl", "reference", "--steps", "2", "--warmup", "3")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["dtype"] == "f64"
    assert d["config"]["workload"] == bench.WORKLOAD and d["data"] == "synthetic"
    assert d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    p = _run("--impl", "reference", "--steps", "1", "--warmup", "3",
             env={"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_fewer_than_three_warmup_steps_are_refused():
    p = _run("--impl", "reference", "--steps", "1", "--warmup", "2")
    assert p.returncode == 2 and "--warmup must be >= 3" in p.stderr


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c


OK = "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"
CAPPED = "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
HOT = "0, 1500, 2070, 1200.0, 0x20, Not Active, Active, Not Active, Not Active"


def test_clock_record_reads_the_timed_region():
    c = _sampler([(0.5, HOT), (1.0, OK), (1.1, CAPPED), (1.2, OK), (1.3, "[Unknown Error]"),
                  (3.0, HOT)])
    s = c.summary(1.0, 2.0)
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    # no sample inside the window: the whole run is summarised, and says so
    s = c.summary(5.0, 6.0)
    assert s["samples"] == 5 and s["sm_mhz"] == 1900.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["window"].startswith("whole sampler run")


def test_clock_record_without_nvidia_smi():
    s = _sampler([]).summary(0.0, 1.0)
    assert s["samples"] == 0 and s["reasons"] == ["nvidia-smi unavailable"]
    assert s["sm_mhz"] is None


def test_relative_error_summary():
    oc = np.array([10.0, 20.0, np.inf, 40.0])
    c = np.array([10.0, 20.002, np.inf, np.inf])
    out = bench._rel(c, oc)
    assert out["sample"] == 4 and out["infeasible_differ"] == 1
    assert out["max_rel_err"] == pytest.approx(1e-4, rel=1e-9)
    assert out["mean_rel_err"] == pytest.approx(5e-5, rel=1e-9)
    # the means of the scenarios finite on both sides: 15.001 against 15
    assert out["rel_err_of_mean"] == pytest.approx(0.001 / 15.0, rel=1e-9)


def test_split_errors_compare_predecessors_at_unique_optima_only():
    orc = {"cost": np.array([5.0, 6.0]),
           "pred": np.array([[0, 1, 1], [0, -1, -1]], np.int32),
           "margin": np.array([[1.0, 1e-6, 0.5], [1.0, np.inf, np.inf]])}
    cost = np.array([5.0, 6.0], np.float32)
    pred = np.array([[0, 0, 1], [0, 3, 3]], np.int64)  # differs only at a near-tie
    out = bench.split_errors(cost, pred, orc)           # and past an infeasible position
    assert out["pred_checked"] == 3 and out["pred_mismatch"] == 0
    assert out["max_rel_err"] == 0.0
    pred[0, 2] = 0
    assert bench.split_errors(cost, pred, orc)["pred_mismatch"] == 1
    assert "pred_checked" not in bench.split_errors(cost, None, orc)


def test_reinsert_errors_follow_the_oracle_path():
    U, I0 = 10, 5
    cons = np.array([[3, 4, 2]])
    op = np.array([[1, 0, 1]], np.uint8)  # states on the path: 5, then 10 - 3 = 7, then 3
    margin = np.ones((1, 3, U + 1))
    orc = {"value": np.array([12.0]), "policy": op, "margin": margin}
    val = np.array([12.0], np.float32)
    out = bench.reinsert_errors(val, op.copy(), orc, cons, U, I0)
    assert (out["policy_checked"], out["policy_mismatch"]) == (3, 0)
    bad = op.copy()
    bad[0, 0] = 0                                       # a clear decision taken wrongly
    out = bench.reinsert_errors(val, bad, orc, cons, U, I0)
    assert (out["policy_checked"], out["policy_mismatch"]) == (3, 1)
    margin[0, 1, 7] = 1e-7                              # a near-tie on the path at day 1
    out = bench.reinsert_errors(val, op.copy(), orc, cons, U, I0)
    assert (out["policy_checked"], out["policy_mismatch"]) == (2, 0)
    tie = op.copy()
    tie[0, 1] = 1                                       # the other side of the tie: the
    out = bench.reinsert_errors(val, tie, orc, cons, U, I0)  # paths part, the scenario stops
    assert (out["policy_checked"], out["policy_mismatch"]) == (1, 0)


@pytest.mark.parametrize("name", ["split_pipe_traffic.json", "split_deque_traffic.json"])
def test_traffic_records_scale_their_capture(name):
    with open(os.path.join(ROOT, "profiles", name)) as f:
        tj = json.load(f)
    want = ((tj["dram_bytes_read_captured"] + tj["dram_bytes_write_captured"])
            * tj["scaled_to_scenarios"] / tj["captured_scenarios"])
    assert tj["dram_bytes_per_launch"] == pytest.approx(want, rel=1e-12)
    assert tj["scaled_to_scenarios"] == 1_000_000
    assert "--clock-control none" in tj["command"] and "python bench.py" in tj["command"]
    assert len(tj["kernel_rev"]) == 16


def test_kernel_rev_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    with open(os.path.join(ROOT, "paper_2602_05179_gb300", "csrc", "split_pipe.cu")) as f:
        src = f.read()
    d = tmp_path / "paper_2602_05179_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "split_pipe.cu").write_text(src)
    h0 = bench.kernel_rev("pipe")
    (d / "split_pipe.cu").write_text("// a new comment\n\n" + src.replace("\n", "  // note\n", 1))
    assert bench.kernel_rev("pipe") == h0
    assert "kCheckEvery = 2;" in src
    (d / "split_pipe.cu").write_text(src.replace("kCheckEvery = 2;", "kCheckEvery = 4;"))
    assert bench.kernel_rev("pipe") != h0


def test_reference_arm_under_torchrun_prints_one_line():
    """Launched as the N > 1 runs are (torchrun, one process per rank, the
    rendezvous on 127.0.0.1): rank 0 alone runs the oracle and prints the one
    JSON line; the other rank exits 0 without output."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0

"""Host side of the benchmark (no GPU): the roofline's algorithmic bytes
per launch, the rule that recorded ncu counters are used only for the
kernel code they were taken on, the config both arms name, and the
reference arm (the oracle on the host cores) run end to end."""
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNELS = os.path.join(ROOT, "paper_2207_07615_gb300", "csrc", "plss_kernels.cu")


def test_algorithmic_bytes_of_the_c2_sweeps():
    """Each array touched once: CSR or CSC (int32 index + value per nonzero,
    int32 offsets), the gathered vector once, the written vectors once."""
    m, n, nnz = 1_000_000, 200_000, 8_000_000
    assert bench.sweep_bytes("row_sweep", m, n, nnz, 8) == nnz * 12 + (m + 1) * 4 + 2 * m * 8 + n * 8
    assert bench.sweep_bytes("row_sweep", m, n, nnz, 8) == 117_600_004
    assert bench.sweep_bytes("col_sweep", m, n, nnz, 8) == 106_400_004
    assert bench.sweep_bytes("update", m, n, nnz, 8) == 8_000_000
    assert bench.sweep_bytes("row_sweep", m, n, nnz, 4) == nnz * 8 + (m + 1) * 4 + 2 * m * 4 + n * 4
    with pytest.raises(KeyError):
        bench.sweep_bytes("other", m, n, nnz, 8)


def _tree(tmp_path, kernels_text, traffic_text):
    csrc = tmp_path / "paper_2207_07615_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "plss_kernels.cu").write_text(kernels_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(traffic_text)
    return str(tmp_path)


def test_counters_follow_the_sweep_code(tmp_path, monkeypatch):
    src = open(KERNELS, encoding="utf-8").read()
    traffic = open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")).read()
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "a", src, traffic))
    assert bench.ncu_traffic("col_sweep") == 113637120.0     # the committed record matches the source
    # a comment edit keeps the counters
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "b", "// note\n" + src.replace(
        "namespace plss {", "namespace plss {  // edited comment", 1), traffic))
    assert bench.ncu_traffic("col_sweep") == 113637120.0
    # a code change in the grid sweeps voids them
    body = src.replace("constexpr int kBatch = 8;", "constexpr int kBatch = 4;", 1)
    assert body != src
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "c", body, traffic))
    assert bench.ncu_traffic("col_sweep") is None
    # a change confined to the cluster solver keeps them
    cl = src.replace("constexpr int kClusterThreads = 512;", "constexpr int kClusterThreads = 256;", 1)
    assert cl != src
    monkeypatch.setattr(bench, "ROOT", _tree(tmp_path / "d", cl, traffic))
    assert bench.ncu_traffic("col_sweep") == 113637120.0
    # no record: None
    shutil.rmtree(os.path.join(str(tmp_path / "d"), "profiles"))
    assert bench.ncu_traffic("col_sweep") is None


def test_both_arms_name_the_same_config():
    """The reference arm's line carries the GPU arm's config dict."""
    import argparse
    args = argparse.Namespace(prec="fp64", tol=1e-8, w_mode=0)
    a = bench.run_config(args, 1_000_000, 200_000, 8_000_000, 1)
    b = bench.run_config(args, 1_000_000, 200_000, 8_000_000, 1)
    assert a == b and a["workload"] == bench.WORKLOAD and a["parallelism"] == "single"
    assert "224 MB" in a["l2"]
    assert bench.run_config(args, 1_000_000, 200_000, 8_000_000, 4)["parallelism"] == "replicas"


def _run_bench(*argv, env_extra=None):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_line_of_the_contract():
    """The reference arm (the oracle, host cores only) runs without a GPU:
    one JSON line with the GPU arm's metric, unit, direction and config, a
    cpu_baseline describing the run, and an e2e object with no copies."""
    (line,) = _run_bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["steps"] == 1 and line["warmup"] == 0
    assert line["n_gpus"] == 1 and line["data"] == "synthetic" and line["dtype"] == "f64"
    assert line["config"]["workload"] == bench.WORKLOAD and line["config"]["nnz"] == 8_000_000
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "100 updates" in cb["sample"] and str(bench.REF_UPDATES_TO_TOL) in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # an update of the oracle costs milliseconds, so the extrapolated solve is hours, not zero
    assert line["value"] > bench.REF_UPDATES_TO_TOL * 1e-4


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle; the others print nothing."""
    assert _run_bench("--impl", "reference", "--steps", "1", "--warmup", "0",
                      env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_clock_record_from_sampled_rows(tmp_path, monkeypatch):
    """The clocks key: median SM clock over the samples drawn under load
    (power at or above the median), the maximum clock, and every throttle
    reason seen Active -- here from a stand-in nvidia-smi that prints three
    rows in the queried column order and waits to be stopped."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "printf '2070, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active\\n'\n"
                    "printf '1900, 2070, 720.0, 0x4, Not Active, Not Active, Not Active, Active\\n'\n"
                    "printf '1500, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active\\n'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    time.sleep(0.5)
    rec = c.stop()
    assert rec == {"sm_mhz": 1985.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                   "power_w_max": 720.0}


def test_clock_record_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    assert bench.Clocks(0).stop() is None

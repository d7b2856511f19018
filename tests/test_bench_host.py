"""Host-side arithmetic of the benchmark's roofline (no GPU): the
algorithmic bytes per launch, and the rule that recorded ncu counters are
used only for the kernel code they were taken on."""
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

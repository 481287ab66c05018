"""The benchmark's output contract, on the CPU: the reference arm (the FP64
oracle timed on the host cores) prints one JSON line with the required keys,
and the helpers that attach DRAM traffic and the run log behave."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


REQUIRED = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
            "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
            "config": dict}


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k, t in REQUIRED.items():
        assert isinstance(d[k], t), k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GD/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    one = d["cpu_baseline"]["one_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": "GD/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_recorded_traffic_parser(tmp_path, monkeypatch):
    h = bench.tc_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(
        "text\n`traffic-record: kernel=k_gemm1_tc workload=96^3/4096/K16/bf16x3 shape=g1_nb=256,g1_dpt=1 "
        f"source_sha256={h} dram_bytes_per_launch=123.0`\n"
        "`traffic-record: kernel=k_gemm1_tc workload=96^3/4096/K16/bf16x3 shape=g1_nb=128,g1_dpt=2 "
        "source_sha256=0000 dram_bytes_per_launch=5`\n"
        "`tensor-pipe-record: kernel=k_gemm2_tc workload=96^3/4096/K16/bf16x3 shape=g2_bn=256,g2_kgroup=4 "
        f"source_sha256={h} pct_of_elapsed=81.5`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "tc_source_hash", lambda: h)
    assert bench.recorded_traffic("k_gemm1_tc", "96^3/4096/K16/bf16x3", "g1_nb=256,g1_dpt=1") == 123.0
    # a record taken with other kernel sources, or another shape, is not used
    assert bench.recorded_traffic("k_gemm1_tc", "96^3/4096/K16/bf16x3", "g1_nb=128,g1_dpt=2") is None
    assert bench.recorded_traffic("k_gemm2_tc", "96^3/4096/K16/bf16x3", "g1_nb=256,g1_dpt=1") is None
    assert bench.recorded_tensor_pipe("k_gemm2_tc", "96^3/4096/K16/bf16x3", "g2_bn=256,g2_kgroup=4") == 81.5
    assert bench.recorded_tensor_pipe("k_gemm1_tc", "96^3/4096/K16/bf16x3", "g1_nb=256,g1_dpt=1") is None
    assert bench.recorded_traffic("k_gemm2_tc", "96^3/4096/K16/bf16x3", "g2_bn=256,g2_kgroup=4") is None


def test_run_log_and_context(tmp_path):
    p = tmp_path / "runs.jsonl"
    bench.append_jsonl(str(p), {"metric": bench.METRIC, "value": 1.0})
    bench.append_jsonl(str(p), {"metric": bench.METRIC, "value": 2.0})
    recs = [json.loads(ln) for ln in p.read_text().splitlines()]
    assert [r["value"] for r in recs] == [1.0, 2.0]
    assert all("time_utc" in r and r["host"]["cores"] >= 1 for r in recs)
    assert abs(sum(bench.kp_weights(bench.KP_NK)) - 1.0) < 1e-15
    assert "3.4x" in bench.PAPER_CONTEXT["scf_cost_reduction_vs_kerker"]


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the multi-GPU runs are (torchrun, 2 ranks, 127.0.0.1): rank
    0 alone times the oracle and prints the one JSON line, the other rank
    exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29517", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    # torchrun's one OpenMP thread per rank does not throttle the only working rank
    assert d["cpu_baseline"]["cores"] == os.cpu_count()

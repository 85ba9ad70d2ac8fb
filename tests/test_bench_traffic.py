"""bench.py reports the ncu DRAM traffic of the dominant kernel only while the
kernel sources still match the ones the counters were taken from (stale
counters read as null)."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_traffic_matches_the_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic_per_launch.json")))
    for kernel in (bench.COST["classic"]["kernel"], bench.COST["newcg"]["kernel"]):
        assert kernel in d, kernel
        t = bench.captured_traffic(kernel)
        assert t is not None and t > 0, kernel
        # per-launch bytes of the 500-iteration benchmark, close to its algorithmic minimum
        alg = d[kernel]["algorithmic_bytes_per_iteration"] * bench.ITERS
        assert 0.5 * alg < t < 1.5 * alg


def test_stale_sources_give_no_traffic(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    shutil.copytree(os.path.join(ROOT, "paper_1803_03797_gb300", "csrc"), root / "paper_1803_03797_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    kernel = bench.COST["newcg"]["kernel"]
    assert bench.captured_traffic(kernel) is not None
    with open(root / "paper_1803_03797_gb300" / "csrc" / "cg_kernels.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.captured_traffic(kernel) is None
    assert bench.captured_traffic("k_unknown<double,2>") is None

"""bench.py's reference arm (the CPU oracle, as the driver launches it) prints the one JSON line
the contract asks for (CPU only: a tiny sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-waveforms", "64",
                          "--mcmc-steps", "50", "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "batched_uneven_100k"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]



def test_capture_data_is_taken_only_for_its_kernel_source_and_workload(tmp_path, monkeypatch):
    """roofline.traffic and roofline.issue come from a committed ncu capture of the same kernel
    source and the same workload; another workload, or a changed source, gets nothing."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cuh"
    src.write_bytes(b"// a kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    entry = {"warp_inst_per_step": 100.0, "traffic_bytes_per_launch": 10, "units_per_launch": 5, "units": "steps"}
    (tmp_path / "profiles" / "k_dram_traffic.json").write_text(
        json.dumps({"kernel_sha": sha, "workloads": {"w1": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic(str(src), "k", "w1") == entry
    assert bench.load_traffic(str(src), "k", "w2") is None
    src.write_bytes(b"// a changed kernel source\n")
    assert bench.load_traffic(str(src), "k", "w1") is None
    assert bench.load_traffic(str(src), "absent", "w1") is None


def test_committed_capture_covers_the_default_workload():
    """The committed capture of the PE kernel (when it is of the current source) has the default
    workload's warp instructions per step and DRAM bytes per launch."""
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2403_03156_gb300", "csrc", "fsmp_pe_kernel.cuh")
    d = bench.load_traffic(src, "pe_kernel", "batched_uneven_100k")
    if d is None:
        pytest.skip("the committed capture predates the current kernel source")
    assert d["warp_inst_per_step"] > 0 and d["traffic_bytes_per_launch"] > 0 and d["units_per_launch"] > 0

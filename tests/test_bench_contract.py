"""The bench's reference arm (the CPU oracle) keeps the one-JSON-line
contract; it needs no GPU, so it runs here."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, str(ROOT / "bench.py"), *args], cwd=ROOT, env=e, capture_output=True,
                          text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run_bench("--impl", "reference", "--config", "1", "--steps", "2", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 0
    assert d["unit"] == "packets/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"].startswith("packets/s") and d["data"] == "synthetic"
    assert d["ms_per_step"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = run_bench("--impl", "reference", "--config", "1", "--steps", "1", "--warmup", "0",
                  env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_traffic_record_follows_the_kernels_code(tmp_path, monkeypatch):
    """The DRAM-traffic figures bench.py reports apply to one build of the
    kernels: its fingerprint ignores comments and blank lines but changes
    with any code change."""
    sys.path.insert(0, str(ROOT))
    import bench
    csrc = tmp_path / "paper_2510_14050_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ans_x.cu").write_text("// header\n__global__ void k(int* p) { p[0] = 1; }  // store\n")
    (csrc / "ans_x.cuh").write_text("#pragma once\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.library_fingerprint()
    (csrc / "ans_x.cu").write_text("/* reworded\n   header */\n\n__global__ void k(int* p) { p[0] = 1; }\n")
    assert bench.library_fingerprint() == a
    (csrc / "ans_x.cu").write_text("__global__ void k(int* p) { p[0] = 2; }\n")
    assert bench.library_fingerprint() != a
    rec = bench.NCU_TRAFFIC[bench.DEFAULT_CONFIG]
    assert rec["step"] > 0 and all(v > 0 for v in rec["kernels"].values())

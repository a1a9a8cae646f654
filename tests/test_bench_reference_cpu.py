"""The reference arm of the benchmark (the CPU oracle timed on the host) and
its JSON line: run as a subprocess on the Chung-Lu workload, one step, no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "chung_lu", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "chung_lu_n200k_m2M_gamma2.5_h2_h3"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_table_lines(tmp_path, monkeypatch):
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_per_launch.txt").write_text(
        "# comment\nwl_a levelU ratio 0.5\nwl_a bfs 1234.5\nwl_b levelU 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("wl_a", "levelU", 1000.0) == 500.0  # ratio x algorithmic bytes
    assert bench.profile_traffic("wl_a", "bfs", 1000.0) == 1234.5    # bytes per launch
    assert bench.profile_traffic("wl_b", "levelU", 1000.0) == 99.0
    assert bench.profile_traffic("wl_a", "peel", 1000.0) is None


def test_committed_traffic_line_is_the_levelU_ratio():
    import bench
    wl = bench.Workload("rmat")
    assert bench.profile_traffic(wl.name, "levelU", 1e8) == 0.52 * 1e8

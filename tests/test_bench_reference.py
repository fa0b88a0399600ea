"""The CPU reference arm of bench.py (the oracle timed on the host cores) prints
one well-formed JSON line with the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--cpu-budget", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "WL flip attempts/s" and d["unit"] == "attempts/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("2D Ising REWL batch")


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_stage_table_reads_per_window_stage_ends():
    """Per stage: the sweeps each window took (mean and largest over the
    windows of all instances) and when the stage's last window ended it."""
    import numpy as np
    bench = _bench()
    a = np.full((2, 33), -1, np.int64)
    a[:, 0] = [10, 30]
    a[:, 1] = [25, 50]
    b = np.full((2, 33), -1, np.int64)
    b[:, 1] = [40, 44]               # a warm start that began at stage 1
    rows = bench._stage_table([a, b])
    assert [r["stage"] for r in rows] == [0, 1]
    assert rows[0]["mean_window_sweeps"] == 20 and rows[0]["max_window_sweeps"] == 30
    assert rows[0]["last_window_end"] == 30
    # stage 1: 15, 20 (instance a), 40, 44 (instance b, counted from 0)
    assert rows[1]["mean_window_sweeps"] == (15 + 20 + 40 + 44) / 4 and rows[1]["max_window_sweeps"] == 44
    assert rows[1]["last_window_end"] == (50 + 44) / 2


def test_profile_fields_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    bench = _bench()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "sweep_kernel_ising_config1.md").write_text(
        "traffic_bytes_per_launch_full: 37122560\nmeasured_issue_lane_slots_per_trial: 421.9\n"
        "issue_slots_active_pct: 31.1\nsource_sha256: abc123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profile_fields("abc123") == {"traffic": 37122560.0, "instr_per_trial_measured": 421.9,
                                               "issue_slots_active_pct": 31.1}
    assert bench._profile_fields("def456") == {}


def test_restricted_energy_range_instances():
    from paper_1407_5140_gb300 import workloads as W
    ds = W.potts_fss(sizes=(200,), seeds=2, walkers=1, e_range=(-1.9, -0.7))
    assert len(ds) == 2 and ds[0]["seed"] != ds[1]["seed"]
    assert ds[0]["e_min"] == -76000 and ds[0]["e_max"] == -28000
    # about 490-bin windows at 75 % overlap over 48001 bins
    assert ds[0]["n_windows"] == 389
    full = W.potts_fss(sizes=(100,), seeds=1, walkers=1)[0]
    assert (full["e_min"], full["e_max"], full["n_windows"]) == (-20000, 0, 160)

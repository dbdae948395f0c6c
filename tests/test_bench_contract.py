"""The bench's reference arm (the CPU oracle) runs without a GPU: its JSON
line carries the contract's keys, for a small lattice."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    t0 = time.time()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0", "--lattice", "4,4,4,8"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    wall = time.time() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 0
    # the claimed timed region fits inside the process's own run time
    assert d["steps"] * d["ms_per_step"] / 1000.0 < wall
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("4^3x8 staggered")
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the projection from a bounded sample, checked against complete solves
    pc = d["projection_check"]
    for name in ("all_cores", "one_core"):
        c = pc[name]
        assert c["iters"] > 0 and c["full_solve_s"] > 0 and c["projected_s"] > 0
        assert 0.2 < c["full_over_projected"] < 5.0
    # one complete solve of the workload, measured
    fs = d["full_solve"]
    assert fs["seconds"] > 0 and fs["iters"] > 0 and fs["true_res"] <= 1e-10


def test_oracle_workload_json_line():
    """The reference arm's `--workload oracle` times the CPU oracle's Dslash
    and A (host cores only, no GPU) per configuration lattice; without
    `--impl reference` the workload is refused."""
    bench = os.path.join(ROOT, "bench.py")
    r = subprocess.run([sys.executable, bench, "--workload", "oracle", "--oracle-configs", "c1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode != 0 and "--impl reference" in r.stderr
    r = subprocess.run([sys.executable, bench, "--impl", "reference", "--workload", "oracle",
                        "--oracle-configs", "c1,c2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert d["impl"] == "reference" and d["kind"] == "oracle" and d["cores"] >= 1
    assert [row["config"] for row in d["rows"]] == ["c1", "c2"]
    for row in d["rows"]:
        for op in ("dslash", "apply_A"):
            for where in ("all_cores", "one_core"):
                assert row[f"{op}_{where}_ms"] > 0 and row[f"{op}_{where}_gbs"] > 0
    c2 = d["rows"][1]
    assert c2["lattice"] == "16x16x16x32" and c2["vh"] == 16 * 16 * 16 * 32 // 2

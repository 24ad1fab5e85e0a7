"""bench.py's host logic on the CPU: the reference arm's JSON line (the oracle timed on the
host), its rank rule under torchrun, the compulsory-byte model, and the recorded DRAM traffic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
           "--steps", "3", "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_line():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_compulsory_bytes_closed_forms():
    # 12 B per nonzero (value + column), 4 (m + 1) row pointers, x read once, y written once
    n27 = (3 * 100 - 2) ** 3  # 27-point stencil on 100^3: (3N - 2)^3 nonzeros
    assert n27 == 26_463_592
    assert bench.compulsory_bytes(10**6, 10**6, n27, 1) == 337_563_108
    assert bench.compulsory_bytes(2 * 10**6, 2 * 10**6, 10**8, 1) == 1_240_000_004
    # SpMM: X and Y move k values per row
    assert bench.compulsory_bytes(10, 20, 30, 4) == 12 * 30 + 4 * 11 + 8 * 20 * 4 + 8 * 10 * 4


def test_recorded_traffic_is_plausible():
    """Every recorded DRAM figure names a kernel variant (with rN for a relabelling plan), a
    16-hex-digit source hash and a benchmark matrix, and lies within 10 % of that matrix's
    compulsory bytes (more would mean re-reads)."""
    sizes = {"stencil3d_100": (10**6, 10**6, 26_463_592), "banded_2M_hbw1000_50": (2 * 10**6, 2 * 10**6, 10**8)}
    seen = 0
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        assert f[0].split("r")[0] in ("1", "2", "3", "4", "5")
        assert f[0] == bench.traffic_key(int(f[0].split("r")[0]), int(f[0].split("r")[1]) if "r" in f[0] else 0)
        assert len(f[1]) == 16 and int(f[1], 16) >= 0
        if f[3] in sizes:
            cb = bench.compulsory_bytes(*sizes[f[3]], 1)
            assert 0.9 * cb <= float(f[2]) <= 1.1 * cb, line
            seen += 1
    if seen == 0:
        pytest.skip("no stencil or banded entry recorded")

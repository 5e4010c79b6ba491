"""bench.py's output contract, checked on the CPU: the reference arm (the
FP64 oracle on the host) prints one JSON line with the keys the driver
reads, and the helpers that combine ranks behave."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "unit_cube_20", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d) and d["impl"] == "reference"
    assert d["metric"] == "tet-element updates/s" and d["unit"] == "tet-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "unit_cube_20"


def test_rank_helpers_single_process():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    # whole-job throughput: units of all ranks over the slowest rank's time
    assert bench.job_throughput(1000, 10, 4, 2.0) == pytest.approx(1000 * 10 * 4 / 2.0)


def test_traffic_record_names_the_digest_sources():
    """The DRAM-traffic record lists the sources whose digest it carries,
    the same ones bench.py hashes, and each entry's digest is a SHA-256
    (bench.py reports the traffic only while the digest matches)."""
    import bench
    with open(bench.TRAFFIC_FILE) as fh:
        rec = json.load(fh)
    assert tuple(rec["sources"]) == bench.TRAFFIC_SOURCES
    for f in bench.TRAFFIC_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1005_3158_gb300", "csrc", f)), f
    for e in rec["entries"]:
        assert len(e["sources_sha256"]) == 64 and e["units"] > 0
        assert e["dram_read_bytes"] > 0 and e["dram_write_bytes"] > 0

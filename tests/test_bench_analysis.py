"""bench.py --analysis-only: the host analysis timed alone, without a GPU.

The mode runs glu_analyze with host_only (the fill, Algorithm 4, the levels
and the schedules on the host cores) and prints one JSON line; its counts
must be the analysis's own (the oracle's fill size and level count for the
32 x 32 grid in natural order, the workload the survey pins: 64,574 entries
of L+U, 1,024 levels)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--analysis-only", "grid32_natural",
                          "--steps", "2", *extra], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_analysis_only_line():
    d = run()
    assert d["metric"] == "host analysis time" and d["workload"] == "grid32_natural"
    assert d["n"] == 1024 and d["nnz_lu"] == 64574 and d["nlevels"] == 1024
    assert len(d["analyze_s"]) == 2 and all(t > 0 for t in d["analyze_s"])
    assert d["analyze_s_median"] > 0 and d["factor_blocks"] == 0


def test_analysis_only_supernodal():
    d = run("--factor-blocks")
    assert d["factor_blocks"] == 1 and d["nnz_lu"] == 64574

"""Allocation failures in the host analysis (no GPU).

The analysis builds the column schedule on worker threads and the solve
schedule on a thread of its own.  A failed allocation on any of them must
come back as GLU_ERR_OOM from glu_analyze, with every thread joined and the
process intact; the next analysis must then run normally.  The failures are
made on the host: two test hooks make one level of the column schedule, or the
solve schedule, fail as an allocation would, and a subprocess runs the
analysis under an address-space limit too small for it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from paper_1908_00204_gb300 import glu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mat():
    return synth.make("mesh100x200_nets64", 1)


def analyze(m):
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1))
    try:
        return glu.glu_get_levels(h), glu.glu_get_stats(h)["nlevels"]
    finally:
        glu.glu_destroy(h)


@pytest.mark.parametrize("where", ["first", "last"])
def test_schedule_level_failure_reports_oom(mat, monkeypatch, where):
    (lp0, lc0), nl = analyze(mat)
    # four threads take ranges of levels as they finish: the failing level
    # may be scheduled on the calling thread or on a worker
    monkeypatch.setenv("GLU_ANALYZE_THREADS", "4")
    monkeypatch.setenv("GLU_TEST_FAIL_LEVEL", "0" if where == "first" else str(nl - 1))
    with pytest.raises(glu.GluError) as e:
        analyze(mat)
    assert e.value.code == glu.GLU_ERR_OOM
    monkeypatch.delenv("GLU_TEST_FAIL_LEVEL")
    (lp, lc), _ = analyze(mat)
    assert np.array_equal(lp, lp0) and np.array_equal(lc, lc0)


def test_solve_schedule_failure_reports_oom(mat, monkeypatch):
    monkeypatch.setenv("GLU_TEST_FAIL_SOLVE", "1")
    with pytest.raises(glu.GluError) as e:
        analyze(mat)
    assert e.value.code == glu.GLU_ERR_OOM
    monkeypatch.delenv("GLU_TEST_FAIL_SOLVE")
    analyze(mat)


PROBE = r"""
import resource, sys
sys.path.insert(0, {root!r})
import synth
from paper_1908_00204_gb300 import glu
m = synth.make("mesh100x200_nets64", 1)
glu.default_options()          # loads the library before the limit
for line in open("/proc/self/status"):
    if line.startswith("VmSize"):
        lim = int(line.split()[1]) * 1024 + (60 << 20)
resource.setrlimit(resource.RLIMIT_AS, (lim, lim))
try:
    glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1))
    print("ok")
except glu.GluError as e:
    print("code", e.code)
"""


def test_address_space_limit_reports_oom():
    env = dict(os.environ, GLU_ANALYZE_THREADS="1")
    r = subprocess.run([sys.executable, "-c", PROBE.format(root=ROOT)], capture_output=True, text=True,
                       timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == f"code {glu.GLU_ERR_OOM}"

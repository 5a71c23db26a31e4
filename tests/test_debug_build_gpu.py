"""The bounds-checked build (CHER_DEBUG): every table, grid, record,
trace, shared-memory and fallback-queue index of the kernels is checked
before its access; a failed check sets a bit of stats[CHER_STAT_DEBUG],
which cher_sync_status reports as CHER_EBOUNDS, and the access is moved
inside its array (nothing traps).  The small parity cases run through that
build in a process of their own and must pass unchanged: every launch
status they check would read CHER_EBOUNDS if any index had left its array.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_parity_cases_through_the_bounds_checked_build():
    from paper_2006_14927_gb300.build import OUT_DEBUG, build
    assert build(debug=True) == OUT_DEBUG
    env = dict(os.environ, CHER_DEBUG="1")
    which = subprocess.run([sys.executable, "-c",
                            "import paper_2006_14927_gb300 as P; print(P.LIB_PATH)"],
                           env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert which.returncode == 0 and which.stdout.strip() == OUT_DEBUG, which.stderr
    cases = ("plain_fp64_workload or vertical_shower_reduced or inclined_shower_large_tables or "
             "launch_shapes or track_base or edge_cases or overflow_writes or "
             "library_refuses or many_tiles")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_parity_gpu.py"), "-k", cases],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout

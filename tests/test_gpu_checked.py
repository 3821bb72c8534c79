"""The bounds-checked build (ATOS_CHECKED) on the parity suite: in place of compute-sanitizer, the
worker engines, task bodies and level-synchronous kernels check every popped item, CSR entry
index, neighbour id and push-buffer slot, and record a violation as ATOS_ERR_BOUNDS (with its
site) instead of touching memory outside the arrays.  tests/checked_suite.py runs the small-graph
suite on that library in a subprocess: every case must match the oracle with no violation, and a
planted out-of-range column index must be caught by the device checks."""
import json
import os
import subprocess
import sys

import pytest

from gpu_common import atos_lib

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_the_parity_suite_without_violations():
    atos_lib()
    from paper_2112_00132_gb300.compile_lib import build
    lib = build(checked=True)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_suite.py"), lib], capture_output=True, text=True,
                       timeout=1200)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert lines, f"no result line:\n{r.stdout[-2000:]}\n{r.stderr[-3000:]}"
    res = json.loads(lines[-1])
    assert res["runs"] > 500
    assert not res["failures"], res["failures"]
    assert res["planted"]["persistent_cta"] == "caught" and res["planted"]["bsp"] == "caught", res["planted"]
    assert res["planted"]["persistent_cta_site"] == 103  # a neighbour id outside [0, n)
    assert r.returncode == 0 and res["ok"]

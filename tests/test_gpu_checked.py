"""The bounds-checked build (-DSS_CHECKED): the library compiled with every
index of the staging, the wide-section search, the learned windows, the
hunt and the global-memory searches checked against its array.  Small plan
cases of every layout and model run against it in a process of their own;
their answers must equal the oracle's and no index may be caught out of
range.  This stands in for a memory checker, which is not available here."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_checked_build_catches_nothing_on_plan_cases():
    from paper_2112_03229_gb300 import _build
    _build.build(checked=True)
    env = dict(os.environ, SS_CHECKED_LIBRARY="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "0 indices out of range" in r.stdout

"""The bounds-checked build (-DKB_CHECKED, the stand-in for a memory checker): built in-tree,
loaded in a child process (KB_CHECKED=1), and run through the gathers, the loop, the vertex
evaluation and both adjoints on ragged and even grids with kb_check_device after every
stage (tests/checked_run.py); the child fails on any skipped out-of-range record access or
on a parity miss against the oracle."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    from paper_2405_20996_gb300 import build as kbuild
    kbuild.build(checked=True)
    env = dict(os.environ, KB_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
    assert "checked run ok" in r.stdout

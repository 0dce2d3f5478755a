"""The debug build (libgtt_debug.so, compiled with -DGTT_DEBUG): every tile
and global index of the kernels is checked against its buffer, and a
violation sets the plan's status word (reported by gtt_plan_check /
gtt_group_check) instead of touching memory outside the buffer.  This runs a
small-case sweep of every kernel family against that build in a child process
(so the release library of this process is not affected) and requires the
status word to stay clear and the results to match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_sweep_keeps_status_clear():
    from paper_2507_02420_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, GTT_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_sweep.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
    assert "status clear" in r.stdout

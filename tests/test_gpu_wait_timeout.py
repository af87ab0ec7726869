"""Failure detection without a GPU fault: every TMA plane wait of the fused step is bounded and,
when it gives up, sets an error bit that lbf_synchronize reports as LBF_EINTERNAL. The LBF_DEBUG
library's probe (include/lbf_debug.h) waits with that same bounded wait on an mbarrier nothing
arrives on (no copy in flight) with a short limit; the status must come back within milliseconds
and the context must keep working."""
import os
import subprocess
import sys

import pytest

from paper_2609_09160_gb300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounded_wait_gives_up_and_reports():
    lib = build.build(debug=True)
    env = dict(os.environ, LBF_LIBRARY=lib, PYTHONPATH=os.pathsep.join([os.path.dirname(HERE), HERE]))
    res = subprocess.run([sys.executable, os.path.join(HERE, "wait_probe.py")], env=env, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0 and res.stdout.startswith("ok"), (res.stdout, res.stderr[-2000:])

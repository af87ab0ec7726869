"""Index checks in place of a memory sanitizer: the LBF_DEBUG build of the library checks every
shared-memory and global index of the fused step against its buffer and reports a violation as
LBF_EINTERNAL (no trap). Every kernel variant (lattice x storage x walls / force field / two
components, TMA and direct loads) runs on odd shapes - single sites, rows shorter than a tile,
ragged tiles in x and y, widths that are and are not TMA-eligible - and must pass every check; the
line-aligned kernel runs the same shapes, and the row split for walls runs channels whose clean run
of rows is long enough for it."""
import os
import subprocess
import sys

import pytest

from paper_2609_09160_gb300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_index_checked_build_passes_on_odd_shapes():
    lib = build.build(debug=True)
    env = dict(os.environ, LBF_LIBRARY=lib, PYTHONPATH=os.pathsep.join([os.path.dirname(HERE), HERE]))
    res = subprocess.run([sys.executable, os.path.join(HERE, "debug_sweep.py")], env=env, capture_output=True,
                         text=True, timeout=1500)
    failed = [l for l in res.stdout.splitlines() if "FAIL" in l]
    assert res.returncode == 0 and not failed, (failed[:10], res.stderr[-2000:])
    assert res.stdout.count(" ok") >= (2 * (4 * 3 + 2 * 1) + 2 * 3 * 3) * 7 + 3 * 4

"""Safety nets of the mining kernel on the GPU, none of which faults it.

* The checking build (TM_CHECK): every data-dependent index into per-warp
  shared memory, the counters, the window table and the tree is checked
  where it is used, and one outside its range becomes TM_ECHECK instead of
  an access.  The parity suite runs once against it: every count must equal
  the oracle's with no check failing.
* A bounded device wait made to run out: in the test build "waits" a warp
  that claimed a donated task gives up on its payload after 16 polls, and
  donors pause about 0.2 ms before publishing.  tm_count must then return
  TM_ETIMEOUT (counts incomplete), the kernel must end by itself, and the
  context must stay usable: the next count on it is exact.

Each runs in a child process that loads the variant library (the binding
loads the library named by TMOTIF_LIB).
"""
import os
import subprocess
import sys

import pytest

from paper_2507_14813_b300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(lib, args, timeout):
    env = dict(os.environ, TMOTIF_LIB=lib, PYTHONPATH=ROOT)
    return subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_parity_suite_under_the_checking_build():
    lib = build.build(variant="check")
    r = _child(lib, ["-m", "pytest", "tests/test_gpu_parity.py", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"],
               timeout=1800)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-2000:])
    assert " passed" in r.stdout and "failed" not in r.stdout


CHILD_WAITS = r"""
import numpy as np
import oracle
from paper_2507_14813_b300 import synth, tmotif
src, dst, t = synth.hub_graph(31, 4000, 40000, 40000)
g = tmotif.Graph(src, dst, t, 4000, presorted=True)
roots = np.nonzero(src == 0)[0][::600].astype(np.int32)        # hub roots: every other warp is idle
ms = [((0, 1), (0, 2), (0, 3), (0, 4)), ((0, 1), (0, 2), (0, 3))]
tr = tmotif.Tree(ms, 2000)
eager = {"ctas_per_sm": 0, "donate_seq": 32, "donate_leaf": 32, "poll_every": 1}
try:
    tmotif.count(g, tr, roots=roots, mode=tmotif.TM_SCHED_DYNAMIC, tune=eager)
    print("RESULT no-timeout")
except tmotif.TMError as e:
    print("RESULT code", e.code)
# the context is usable and the static schedule (no waits) is exact
want = [oracle.count_motif(src, dst, t, m, 2000, roots=roots) for m in ms]
print("RESULT after", tmotif.count(g, tr, roots=roots).tolist() == want)
"""


def test_bounded_wait_runs_out_with_timeout_status():
    lib = build.build(variant="waits")
    r = _child(lib, ["-c", CHILD_WAITS], timeout=600)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-2000:])
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")]
    assert "RESULT code -4" in lines, lines                  # TM_ETIMEOUT
    assert "RESULT after True" in lines, lines

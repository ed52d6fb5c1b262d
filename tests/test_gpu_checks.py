"""The checks build (libemt_checks.so, selected by EMT_CHECKS=1): every
index that comes from device data tested against its array's length, a bad
one latching an error word that emt_sync reports.  The test networks run
under it (in a child process, since a process loads one library) latch no
error and give the same results, bit for bit, as the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
pytestmark = pytest.mark.gpu


def run(checks, path):
    env = dict(os.environ, EMT_CHECKS="1" if checks else "0")
    subprocess.check_call([sys.executable, os.path.join(HERE, "checks_workload.py"), path], env=env, timeout=900)
    return np.load(path)


def test_checks_build_latches_nothing_and_changes_nothing(tmp_path):
    from paper_1903_01081_b300 import build
    build.build(checks=True)
    chk = run(True, str(tmp_path / "checks.npz"))
    ref = run(False, str(tmp_path / "normal.npz"))
    names = [k for k in ref.files if not k.endswith("_status")]
    assert len(names) == 9
    for k in names:
        assert int(chk[k + "_status"][0]) == 0, k
        assert int(ref[k + "_status"][0]) == 0, k
        assert chk[k].size > 0 and np.array_equal(chk[k], ref[k]), k

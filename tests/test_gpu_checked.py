"""The checked build (every data-dependent pool index bounds-checked in the kernels, -DTPC_CHECKED)
on the main workloads, the optional stages and the sweep constructor: no check fires (a failed
check would fail the call with TPC_ERR_CHECK) and the outputs equal the release build's."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1712_09407_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
pytestmark = pytest.mark.gpu


def _run(tmp_path, lib):
    out = str(tmp_path / (os.path.basename(lib) + ".npz"))
    env = dict(os.environ, TPCCA_LIB=lib, PYTHONPATH=os.path.dirname(HERE))
    p = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py"), out], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_runs_clean_and_equals_release(tmp_path):
    checked = build.build(checked=True)
    release = build.build()
    a = _run(tmp_path, checked)
    b = _run(tmp_path, release)
    assert a.keys() == b.keys() and len(a) > 0
    for k in a:
        assert np.array_equal(a[k], b[k]), k

"""The checked build (every index a kernel gathers with is bounds-checked on the device and a
bad one reported as SS_ERR_STATE instead of dereferenced): the Heun, Monte Carlo, midpoint,
semi-implicit, long-row, tensor and demagnetising-field paths run under it without a
violation and give the same results as the normal build (the checks change no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib, out):
    env = dict(os.environ, SPINSYS_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_checked_build_runs_clean_and_matches(tmp_path):
    from paper_1310_6143_gb300 import build as B

    checked = B.build(checked=True)
    normal = B.build()
    a = _run(checked, str(tmp_path / "checked.npz"))
    b = _run(normal, str(tmp_path / "normal.npz"))
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k

"""The oracle built with the benchmark's -O3 flags gives bit for bit the results of an -O2 build:
no optimisation level changes its arithmetic (no FMA contraction, no fast-math), so the CPU
baseline is timed on exactly the program the pins check."""
import os
import subprocess
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib, out):
    env = dict(os.environ, SPINSYS_ORACLE_LIB=lib, PYTHONPATH=ROOT, OMP_NUM_THREADS="2")
    subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_oracle_run.py"), out], check=True, env=env,
                   timeout=600)
    return np.load(out)


def test_o3_build_equals_o2_build(tmp_path):
    o3 = oracle.build()
    o2 = str(tmp_path / "liboracle_o2.so")
    flags = [f if f != "-O3" else "-O2" for f in oracle.FLAGS]
    subprocess.run(["gcc", *flags, "-o", o2, os.path.join(ROOT, "oracle", "spinsys_oracle.c"), "-lm"], check=True)
    a = _run(o3, str(tmp_path / "o3.npz"))
    b = _run(o2, str(tmp_path / "o2.npz"))
    for k in a.files:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)

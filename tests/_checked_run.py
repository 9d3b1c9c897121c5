"""Runs a set of small workloads through the library that SPINSYS_LIB names (the normal or the
checked build) and saves their spins and records to the .npz path given as the argument.  Any
library error (a bounds violation in the checked build reports SS_ERR_STATE) ends it with a
non-zero status.  Used by tests/test_gpu_checked.py only."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1310_6143_gb300 import lattice as L  # noqa: E402
from paper_1310_6143_gb300.system import SpinSystem  # noqa: E402


def main(out):
    res = {}
    sc = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    for prec in ("fp64", "fp32"):
        with SpinSystem(sc, alpha=0.1, dt=1e-16, T=300.0, S0=L.random_state(sc.n, 1), seed=2, precision=prec) as s:
            s.step(50)
            res[f"heun_{prec}"] = s.spins()
            res[f"heun_{prec}_rec"] = s.record(0, 50)
        with SpinSystem(sc, alpha=0.1, dt=1e-16, T=300.0, S0=L.random_state(sc.n, 1), seed=2, precision=prec) as s:
            s.mc_step(20)
            s.midpoint_step(10, iterations=3)
            s.semi_implicit_step(10)
            res[f"alt_{prec}"] = s.spins()
            res[f"alt_{prec}_rec"] = s.record(0, 40)
    lr = L.fcc_long_range(9, 9, 9, r_cut=3.0)
    with SpinSystem(lr, alpha=0.1, dt=1e-16, T=300.0, S0=L.random_state(lr.n, 3), seed=4, precision="fp32") as s:
        assert s.info()["exchange_rows"] == 3
        s.step(20)
        res["rows_packed"] = s.spins()
    lr.J = lr.J * (1.0 + 1e-6 * (np.arange(lr.nnz) % 300))  # more than 255 values: rows read as col + J
    with SpinSystem(lr, alpha=0.1, dt=1e-16, T=300.0, S0=L.random_state(lr.n, 3), seed=4, precision="fp64") as s:
        assert s.info()["exchange_rows"] == 2
        s.step(10)
        res["rows_plain"] = s.spins()
    fcc = L.with_dm(L.fcc(3, 3, 3, with_pos=True), 1e-21)
    fcc.k_c = np.full(fcc.n, 1e-23)
    with SpinSystem(fcc, alpha=0.1, dt=1e-16, T=500.0, S0=L.random_state(fcc.n, 5), seed=6, precision="fp64") as s:
        s.step(20)
        s.mc_step(10)
        res["tensor_mc"] = s.spins()
    a = 3e-10
    pl = L.simple_cubic(8, 8, 3, periodic=(False, False, False), J=6e-21, k_u=1e-23, a=a, with_pos=True)
    with SpinSystem(pl, alpha=0.3, dt=2e-16, T=100.0, S0=L.random_state(pl.n, 7), seed=8, precision="fp64") as s:
        s.set_demag(2 * a, a ** 3, every=5)
        s.step(20)
        s.semi_implicit_step(5)
        res["demag"] = s.spins()
        res["demag_field"] = s.demag_field()
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])

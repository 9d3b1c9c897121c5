"""Child process of test_oracle_build_flags: runs the oracle library named by
SPINSYS_ORACLE_LIB on fixed workloads and saves every result to the .npz given as argv[1]."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle as O  # noqa: E402
from paper_1310_6143_gb300 import lattice as L  # noqa: E402
from tests._helpers import oracle_system  # noqa: E402


def main(path):
    out = {}
    sc = L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24)
    ref = oracle_system(sc, alpha=0.1, dt=1e-16, seed=1)
    out["sc_S"], out["sc_rec"] = O.heun_run(ref, L.uniform_state(sc.n), 60, 300.0, record=True)
    film = L.film(32, 24, 16)
    ref = oracle_system(film, alpha=0.02, dt=1e-16, seed=5)
    T = np.linspace(300.0, 1200.0, 6)
    out["film_S"], out["film_rec"] = O.heun_run(ref, L.random_state(film.n, 3), 6, T, record=True)
    out["gauss"] = O.gaussians_bulk(7, 2, 99, 20000)
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])

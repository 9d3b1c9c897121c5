"""The autotuner's cache (SPINSYS_AUTOTUNE_CACHE): a workload tuned once on a device takes its
stored launch shape without trial runs; another workload gets an entry of its own; the
trajectory does not depend on the tuning."""
import os
import time

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _shape(info):
    return info["exec"], info["block"], info["tile"], info["draw_ahead"]


def test_cache_hit_skips_the_trials(SS, tmp_path):
    path = tmp_path / "tune.txt"
    os.environ["SPINSYS_AUTOTUNE_CACHE"] = str(path)
    try:
        lat = L.simple_cubic(24, 24, 24, J=6e-21, k_u=1e-23)
        S0 = L.random_state(lat.n, 2)
        with SS(lat, T=300.0, S0=S0, seed=4, precision="fp32") as s:
            t0 = time.perf_counter()
            first = s.autotune(4)
            t_first = time.perf_counter() - t0
            s.step(20)
            S_a = s.spins()
        assert len(path.read_text().splitlines()) == 1
        with SS(lat, T=300.0, S0=S0, seed=4, precision="fp32") as s:
            t0 = time.perf_counter()
            second = s.autotune(4)
            t_second = time.perf_counter() - t0
            assert s.step_index == 0
            s.step(20)
            S_b = s.spins()
        assert _shape(second) == _shape(first)
        assert t_second < 0.5 * t_first
        assert np.array_equal(S_a, S_b)
        assert len(path.read_text().splitlines()) == 1
        with SS(L.simple_cubic(25, 24, 24), T=300.0, precision="fp32") as s:
            s.autotune(2)
        assert len(path.read_text().splitlines()) == 2
    finally:
        del os.environ["SPINSYS_AUTOTUNE_CACHE"]

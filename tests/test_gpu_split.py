"""The split FP32-mixed step (a Gaussian pass, then the Heun passes reading it) gives exactly
the fused step's results: the same Gaussians and the same thermal-field products in both
passes.  Checked bit for bit, alone and interleaved with the fused and persistent steps
(whose drawn-ahead Gaussians share the buffer)."""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _run(SS, lats, kw, plan, sched=None):
    """plan: (gaussian_pass, exec, steps) segments."""
    with SS(lats, precision="fp32", **kw) as s:
        if sched is not None:
            s.set_temperature_schedule(sched)
        total = 0
        for gp, ex, k in plan:
            s.set_gaussian_pass(gp)
            s.set_exec(ex)
            assert s.info()["gaussian_pass"] == int(gp)
            s.step(k)
            total += k
        return s.spins(), s.record(0, total), s.magnetisation(), s.energy()


@pytest.mark.parametrize("name", ["film", "fcc", "grains", "core_shell"])
def test_split_step_bitwise_equal_to_fused(SS, name):
    kw = dict(alpha=0.05, dt=1e-16, T=700.0, seed=9)
    if name == "film":
        lats = L.film(40, 36, 16)
    elif name == "fcc":
        lats = L.fcc(5, 6, 5)
    elif name == "core_shell":
        lats = L.core_shell_sphere(diameter=4e-9, r_core=1.5e-9)
        kw["H"] = (1.0, 0.0, 0.0)
    else:
        g, temps = L.grain_ensemble(count=5, n_min=300, n_max=700, layers=3, seed=3)
        lats = g
        kw.update(T=[float(t) for t in temps], seed=[21 + k for k in range(5)])
    fused = _run(SS, lats, kw, [(0, "kernels", 20)])
    split = _run(SS, lats, kw, [(1, "kernels", 7), (1, "graph", 13)])
    conc = _run(SS, lats, kw, [(2, "kernels", 1), (2, "kernels", 6), (2, "graph", 13)])
    mixed = _run(SS, lats, kw, [(0, "kernels", 3), (2, "kernels", 4), (0, "graph", 5), (1, "kernels", 3),
                                (2, "graph", 5)])
    for a, b, c, d in zip(fused, split, conc, mixed):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(a, d)


def test_split_step_under_schedule_and_zero_temperature(SS):
    """A temperature schedule that passes through zero (no Gaussians drawn there) and the
    persistent mode interleaved: still the fused results bit for bit."""
    lat = L.film(24, 20, 8)
    T = np.concatenate([np.full(5, 400.0), np.zeros(6), np.linspace(10.0, 900.0, 30)])
    kw = dict(alpha=0.1, dt=1e-16, T=0.0, seed=4)
    fused = _run(SS, lat, kw, [(0, "kernels", 30)], sched=T)
    split = _run(SS, lat, kw, [(1, "kernels", 9), (1, "persistent", 7), (2, "graph", 14)], sched=T)
    for a, b in zip(fused, split):
        np.testing.assert_array_equal(a, b)


def test_time_passes_reports_the_gaussian_pass(SS):
    with SS(L.film(64, 64, 16), precision="fp32", T=300.0) as s:
        s.set_gaussian_pass(1)
        t = s.time_passes(3)
        assert t["gauss_ms"] > 0 and t["predictor_ms"] > 0 and t["corrector_ms"] > 0
        s.set_gaussian_pass(0)
        assert s.time_passes(2)["gauss_ms"] < t["gauss_ms"]

"""The cluster step of a small single system (one thread-block cluster holding the spins in
shared memory, the Gaussians drawn beforehand, the records summed afterwards) gives the
states and records of the per-step kernels bit for bit, across chunk boundaries, under a
temperature schedule through zero, with per-spin materials, cubic and Neel anisotropy, and in
both precisions; and it refuses what it does not take."""
import numpy as np
import pytest

from paper_1310_6143_gb300 import _binding as B
from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _case(name):
    kw = dict(alpha=0.1, dt=1e-16, T=500.0, seed=5, H=(0.1, -0.2, 0.3))
    if name == "sc10":
        return L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24), kw
    if name == "fcc":
        return L.fcc(4, 4, 4), kw
    if name == "film":
        return L.film(16, 12, 4), kw
    if name == "core_shell":
        return L.core_shell_sphere(diameter=3e-9, r_core=1e-9), dict(kw, H=(1.0, 0.0, 0.0))
    if name == "cubic":
        lat = L.simple_cubic(7, 6, 5, J=6.0e-21, k_u=1.0e-24)
        lat.k_c = np.full(lat.n, 2e-23)
        return lat, kw
    lat = L.simple_cubic(6, 7, 5, periodic=(False, False, False), with_pos=True)
    mask = np.diff(lat.row_ptr) < 6
    lat.K_neel = L.neel_tensors(lat.pos, lat.row_ptr, lat.col, 3e-23, mask)
    return lat, kw


def _run(SS, lat, kw, precision, mode, steps, launch, sched=None):
    with SS(lat, precision=precision, **kw) as s:
        s.set_launch(*launch)
        s.set_exec(mode)
        if sched is not None:
            s.set_temperature_schedule(sched)
        total = 0
        for k in steps:
            s.step(k)
            total += k
        assert s.step_index == total
        return s.spins(), s.record(0, total), s.magnetisation(), s.energy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["sc10", "fcc", "film", "core_shell", "cubic", "neel"])
def test_cluster_step_bitwise_equal_to_kernels(SS, name, precision):
    lat, kw = _case(name)
    for launch in ((128, 256), (256, 256)):
        ref = _run(SS, lat, kw, precision, "kernels", [130], launch)
        got = _run(SS, lat, kw, precision, "cluster", [1, 63, 66], launch)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_step_under_schedule_and_mixed_modes(SS, precision):
    lat, kw = _case("sc10")
    T = np.concatenate([np.full(30, 300.0), np.zeros(50), np.linspace(10.0, 1200.0, 90)])
    kw = dict(kw, T=0.0)
    ref = _run(SS, lat, kw, precision, "kernels", [170], (128, 128), sched=T)
    with SS(lat, precision=precision, **kw) as s:
        s.set_launch(128, 128)
        s.set_temperature_schedule(T)
        for mode, k in (("cluster", 70), ("graph", 20), ("cluster", 45), ("persistent", 10), ("cluster", 25)):
            s.set_exec(mode)
            s.step(k)
        got = (s.spins(), s.record(0, 170), s.magnetisation(), s.energy())
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_cluster_step_refusals(SS):
    small = L.simple_cubic(4, 4, 4)
    with SS([small, small], T=100.0) as s:
        with pytest.raises(B.SpinSysError) as e:
            s.set_exec("cluster")
        assert e.value.status == 7
    with SS(L.simple_cubic(13, 13, 13), T=100.0) as s:  # 2197 spins: more than 2048
        with pytest.raises(B.SpinSysError) as e:
            s.set_exec("cluster")
        assert e.value.status == 7
    with SS(L.fcc_long_range(5, 5, 5, r_cut=2.0), T=100.0) as s:  # rows longer than 12
        with pytest.raises(B.SpinSysError):
            s.set_exec("cluster")

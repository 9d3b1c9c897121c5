"""Slab decomposition of one system on one GPU (Appendix C): K slab handles, each on its own
stream, with device-to-device halo refreshes twice per step, reproduce the undecomposed
handle's spins bit for bit (FP64 and FP32-mixed), because every owned spin draws its thermal
field from the Philox counter of its global index and sums its neighbours in the same order.
The records (eight FP64 sums per step) agree up to the order of the sums."""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L
from paper_1310_6143_gb300 import _binding as B
from paper_1310_6143_gb300.slab import SlabSystem, halo_runs, slab_range

pytestmark = pytest.mark.gpu


def _case(name):
    kw = dict(alpha=0.1, dt=1e-16, T=600.0, seed=7, H=(0.0, 0.2, 0.5))
    if name == "film":
        return L.film(48, 40, 8), kw
    if name == "sc":
        return L.simple_cubic(10, 10, 10), kw
    if name == "fcc":
        return L.fcc(5, 12, 5, J=11.2e-21, k_u=6.69e-24), kw
    lat = L.core_shell_sphere(diameter=4e-9, r_core=1.5e-9)
    kw["H"] = (1.0, 0.0, 0.0)
    return lat, kw


def _whole(lat, kw, precision, plan, sched=None, S_mid=None):
    from paper_1310_6143_gb300.system import SpinSystem

    with SpinSystem(lat, precision=precision, **kw) as s:
        if sched is not None:
            s.set_temperature_schedule(sched)
        total = 0
        for k, steps in enumerate(plan):
            if S_mid is not None and k == 1:
                s.set_spins(S_mid)
            s.step(steps)
            total += steps
        return s.spins(), s.record(0, total)


def _sliced(lat, kw, precision, K, plan, launch=None, sched=None, S_mid=None):
    with SlabSystem(lat, K, precision=precision, **kw) as d:
        if launch:
            d.set_launch(*launch)
        if sched is not None:
            d.set_temperature_schedule(sched)
        total = 0
        for k, steps in enumerate(plan):
            if S_mid is not None and k == 1:
                d.set_spins(S_mid)
            d.step(steps)
            total += steps
        assert d.step_index == total
        return d.spins(), d.record(0, total), d


def _records_close(a, b):
    scale = np.maximum(np.abs(a).max(axis=(0, 1)), 1e-300)
    np.testing.assert_allclose(a / scale, b / scale, rtol=0, atol=1e-11)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["film", "sc", "fcc", "core_shell"])
@pytest.mark.parametrize("K", [2, 3, 4])
def test_slabs_bitwise_equal_to_the_whole_system(name, precision, K):
    lat, kw = _case(name)
    plan = [7, 13]
    S_ref, rec_ref = _whole(lat, kw, precision, plan)
    S, rec, d = _sliced(lat, kw, precision, K, plan, launch=(128, 128))
    if name == "film":  # boundary tiles (the first and last plane), then core tiles
        assert all(0 < s.slab["boundary_tiles"] < s.slab["num_tiles"] for s in d.slabs)
    np.testing.assert_array_equal(S, S_ref)
    _records_close(rec, rec_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_slabs_under_schedule_set_spins_and_default_launch(precision):
    lat, kw = _case("film")
    T = np.concatenate([np.full(4, 300.0), np.zeros(3), np.linspace(50.0, 900.0, 20)])
    S_mid = L.random_state(lat.n, 3)
    kw = dict(kw, T=0.0)
    S_ref, rec_ref = _whole(lat, kw, precision, [5, 9], sched=T, S_mid=S_mid)
    S, rec, _ = _sliced(lat, kw, precision, 3, [5, 9], sched=T, S_mid=S_mid)
    np.testing.assert_array_equal(S, S_ref)
    _records_close(rec, rec_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_slab_random_start_keyed_by_global_index(precision):
    lat, kw = _case("sc")
    kw = dict(kw, init_random=True)
    S_ref, _ = _whole(lat, kw, precision, [0, 4])
    S, _, _ = _sliced(lat, kw, precision, 4, [0, 4])
    np.testing.assert_array_equal(S, S_ref)


def test_slab_handle_runs_and_refusals():
    from paper_1310_6143_gb300.system import SpinSystem

    lat, kw = _case("film")
    K = 3
    for k in range(K):
        with SpinSystem(lat, slab=(K, k), **kw) as s:
            lo, hi = slab_range(lat.n, K, k)
            assert (s.slab["lo"], s.slab["hi"], s.slab["nslabs"], s.slab["slab"]) == (lo, hi, K, k)
            np.testing.assert_array_equal(s.halo_runs(), halo_runs(lat.row_ptr, lat.col, lo, hi))
            assert s.n == hi - lo + s.slab["n_halo"]
            for call in (lambda: s.step(1), lambda: s.mc_step(1), lambda: s.midpoint_step(1),
                         lambda: s.set_demag(1e-9, 1e-29), lambda: s.set_exchange_rows("warp")):
                with pytest.raises(B.SpinSysError) as e:
                    call()
                assert e.value.status == 7
            with pytest.raises(B.SpinSysError):
                s.heun_pass(3, 0, 0)
            with pytest.raises(B.SpinSysError):
                s.heun_pass(0, 0, s.slab["num_tiles"] + 1)
    with pytest.raises(B.SpinSysError):
        SpinSystem(lat, slab=(0, 0), **kw)
    with pytest.raises(B.SpinSysError):
        SpinSystem(lat, slab=(2, 2), **kw)

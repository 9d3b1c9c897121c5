"""Parity of the CUDA midpoint integrator (the midpoint rule the paper's time-integration
section cites as the alternative to Heun; through the C ABI) with the oracle's.

FP64: the same thermal field (same Philox counters), the same Euler predictor and the same
number of fixed-point iterations, so trajectories agree within 1e-12 (sums in a different
order only) and so do the records.  FP32-mixed: 1e-4 over 100 steps.  Steps of the two
integrators share the step counter, the record ring and the temperature schedule.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

pytestmark = pytest.mark.gpu

MU_B = 9.2740e-24


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


@pytest.mark.parametrize("precision,tol,steps,K", [("fp64", 1e-12, 200, 4), ("fp64", 1e-12, 50, 1),
                                                   ("fp32", 1e-4, 100, 4)])
def test_sc_matches_oracle(SS, precision, tol, steps, K):
    lat = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 3)
    H = (0.1, 0.0, 0.4)
    with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, H=H, seed=9, sys_id=2, precision=precision) as s:
        s.midpoint_step(steps, iterations=K)
        S = s.spins()
        rec = s.record(0, steps)
        assert s.step_index == steps
    S_ref, rec_ref = O.midpoint_run(oracle_system(lat, H=H, seed=9, sys_id=2), S0, steps, 300.0, iters=K,
                                    record=True)
    assert np.abs(S - S_ref).max() <= tol
    if precision == "fp64":
        g = rec[:, 0, :]
        assert np.abs(g[:, :4] - rec_ref[:, :4]).max() <= 1e-12 * np.abs(rec_ref[:, 3]).max()
        assert np.abs(g[:, 7] - rec_ref[:, 7]).max() <= 1e-12 * np.abs(rec_ref[:, 7]).max()


def test_fcc_tensor_dm_cubic_and_core_shell_match_oracle(SS):
    lat = L.with_dm(L.fcc(3, 3, 3, J=11.2e-21, k_u=6.69e-24, with_pos=True), 2e-21, (0.0, 0.0, 1.0))
    lat.k_c = np.full(lat.n, 2e-23)
    S0 = L.random_state(lat.n, 5)
    with SS(lat, alpha=0.2, dt=1e-16, T=500.0, S0=S0, seed=4, precision="fp64") as s:
        s.midpoint_step(80, iterations=3)
        S = s.spins()
    ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel, alpha=0.2,
                         dt=1e-16, seed=4, J_tensor=lat.J_tensor, k_c=lat.k_c)
    S_ref, _ = O.midpoint_run(ref, S0, 80, 500.0, iters=3)
    assert np.abs(S - S_ref).max() <= 1e-12
    cs = L.core_shell_sphere(diameter=3.2e-9, r_core=1.2e-9, k_s=5e-23)
    S0 = L.random_state(cs.n, 6)
    with SS(cs, alpha=0.1, dt=1e-16, T=200.0, S0=S0, seed=8, precision="fp64") as s:
        s.midpoint_step(60, iterations=4)
        S = s.spins()
    S_ref, _ = O.midpoint_run(oracle_system(cs, seed=8), S0, 60, 200.0, iters=4)
    assert np.abs(S - S_ref).max() <= 1e-12


def test_batch_and_schedule_equal_each_system_alone(SS):
    lats = [L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23), L.fcc(2, 3, 2), L.simple_cubic(5, 4, 3, J=4e-21)]
    S0s = [L.random_state(l.n, 20 + k) for k, l in enumerate(lats)]
    temps = [300.0, 700.0, 0.0]
    with SS(lats, alpha=0.1, dt=1e-16, T=temps, seed=[1, 2, 3], sys_id=[0, 1, 2], S0=S0s, precision="fp64") as b:
        b.midpoint_step(30, iterations=3)
        S_b = b.spins()
    off = 0
    for k, lat in enumerate(lats):
        S_ref, _ = O.midpoint_run(oracle_system(lat, seed=k + 1, sys_id=k), S0s[k], 30, temps[k], iters=3)
        assert np.abs(S_b[off:off + lat.n] - S_ref).max() <= 1e-12
        off += lat.n
    lat = lats[0]
    T = np.array([0.0, 100.0, 900.0, 300.0, 0.0, 50.0])
    with SS(lat, alpha=0.1, dt=1e-16, T=0.0, S0=S0s[0], seed=4, precision="fp64") as s:
        s.set_temperature_schedule(T)
        s.midpoint_step(len(T), iterations=5)
        S = s.spins()
    S_ref, _ = O.midpoint_run(oracle_system(lat, seed=4), S0s[0], len(T), T, iters=5)
    assert np.abs(S - S_ref).max() <= 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_interleaved_with_heun_shares_the_step_counter(SS, precision, tol):
    """Heun, midpoint, Heun: the thermal field of every step comes from that step's counters
    (Gaussians the FP32 Heun corrector drew ahead for a step the midpoint rule took are not
    reused)."""
    lat = L.simple_cubic(12, 12, 12, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 7)
    with SS(lat, alpha=0.1, dt=1e-16, T=400.0, S0=S0, seed=2, precision=precision) as s:
        s.step(5)
        s.midpoint_step(4, iterations=3)
        s.step(6)
        assert s.step_index == 15
        S = s.spins()
        rec = s.record(0, 15)
    ref = oracle_system(lat, seed=2)
    Sr, r1 = O.heun_run(ref, S0, 5, 400.0, record=True)
    Sr, r2 = O.midpoint_run(ref, Sr, 4, 400.0, iters=3, step0=5, record=True)
    Sr, r3 = O.heun_run(ref, Sr, 6, 400.0, step0=9, record=True)
    assert np.abs(S - Sr).max() <= tol
    if precision == "fp64":
        rr = np.concatenate([r1, r2, r3])
        assert np.abs(rec[:, 0, 7] - rr[:, 7]).max() <= 1e-12 * np.abs(rr[:, 7]).max()


def test_length_is_kept_without_renormalisation(SS):
    """Converged iterations keep |S| = 1 (the rule conserves the length); one iteration does not."""
    lat = L.simple_cubic(8, 8, 8, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 1)
    err = {}
    for K in (1, 10):
        with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=5, precision="fp64") as s:
            s.midpoint_step(100, iterations=K)
            err[K] = np.abs(np.linalg.norm(s.spins(), axis=1) - 1).max()
    assert err[10] < 1e-12 and err[1] > 1e-5


def test_invalid_arguments(SS):
    lat = L.simple_cubic(4, 4, 4, periodic=(False, False, False), with_pos=True)
    with SS(lat, T=0.0) as s:
        for bad in (0, 1001):
            with pytest.raises(Exception, match="iterations"):
                s.midpoint_step(1, iterations=bad)
        with pytest.raises(Exception, match=">= 0"):
            s.midpoint_step(-1)
        s.midpoint_step(2)
        assert s.step_index == 2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_captured_steps_equal_plain_launches(SS, precision):
    """Midpoint steps replayed from captured graphs (a new capture when K changes) equal plain
    launches bitwise, records included."""
    lat = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 12)
    out = {}
    for mode in ("kernels", "auto"):
        with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=6, precision=precision) as s:
            s.set_exec(mode)
            s.midpoint_step(70, iterations=3)
            s.midpoint_step(65, iterations=4)
            s.step(2)
            s.midpoint_step(64, iterations=3)
            out[mode] = (s.spins(), s.record(0, 201))
    assert np.array_equal(out["kernels"][0], out["auto"][0])
    assert np.array_equal(out["kernels"][1], out["auto"][1])

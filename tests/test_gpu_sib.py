"""Parity of the CUDA semi-implicit predictor-corrector (Mentink et al.'s scheme, the modified
predictor-corrector midpoint scheme the paper cites; through the C ABI) with the oracle's.

FP64: the same thermal field (same Philox counters) and the same two closed-form solves, so
trajectories and records agree within 1e-12 (sums in another order only).  FP32-mixed: 1e-4
over 100 steps.  The scheme keeps |S| without renormalisation; its steps share the step
counter, record ring and temperature schedule with the Heun and midpoint steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


@pytest.mark.parametrize("precision,tol,steps", [("fp64", 1e-12, 200), ("fp32", 1e-4, 100)])
def test_sc_matches_oracle(SS, precision, tol, steps):
    lat = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 3)
    H = (0.1, 0.0, 0.4)
    with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, H=H, seed=9, sys_id=2, precision=precision) as s:
        s.semi_implicit_step(steps)
        S = s.spins()
        rec = s.record(0, steps)
        assert s.step_index == steps
    S_ref, rec_ref = O.sib_run(oracle_system(lat, H=H, seed=9, sys_id=2), S0, steps, 300.0, record=True)
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
        s.semi_implicit_step(80)
        S = s.spins()
    ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel, alpha=0.2,
                         dt=1e-16, seed=4, J_tensor=lat.J_tensor, k_c=lat.k_c)
    S_ref, _ = O.sib_run(ref, S0, 80, 500.0)
    assert np.abs(S - S_ref).max() <= 1e-12
    cs = L.core_shell_sphere(diameter=3.2e-9, r_core=1.2e-9, k_s=5e-23)
    S0 = L.random_state(cs.n, 6)
    with SS(cs, alpha=0.1, dt=1e-16, T=200.0, S0=S0, seed=8, precision="fp64") as s:
        s.semi_implicit_step(60)
        S = s.spins()
    S_ref, _ = O.sib_run(oracle_system(cs, seed=8), S0, 60, 200.0)
    assert np.abs(S - S_ref).max() <= 1e-12


def test_batch_schedule_and_interleaving(SS):
    lats = [L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23), L.fcc(2, 3, 2), L.simple_cubic(5, 4, 3, J=4e-21)]
    S0s = [L.random_state(l.n, 20 + k) for k, l in enumerate(lats)]
    temps = [300.0, 700.0, 0.0]
    with SS(lats, alpha=0.1, dt=1e-16, T=temps, seed=[1, 2, 3], sys_id=[0, 1, 2], S0=S0s, precision="fp64") as b:
        b.semi_implicit_step(30)
        S_b = b.spins()
    off = 0
    for k, lat in enumerate(lats):
        S_ref, _ = O.sib_run(oracle_system(lat, seed=k + 1, sys_id=k), S0s[k], 30, temps[k])
        assert np.abs(S_b[off:off + lat.n] - S_ref).max() <= 1e-12
        off += lat.n
    lat = L.simple_cubic(8, 8, 8, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 7)
    T = np.linspace(600.0, 100.0, 20)
    with SS(lat, alpha=0.1, dt=1e-16, T=0.0, S0=S0, seed=2, precision="fp64") as s:
        s.set_temperature_schedule(T)
        s.step(4)
        s.semi_implicit_step(6)
        s.midpoint_step(3, iterations=3)
        s.semi_implicit_step(7)
        assert s.step_index == 20
        S = s.spins()
        rec = s.record(0, 20)
    ref = oracle_system(lat, seed=2)
    Sr, r1 = O.heun_run(ref, S0, 4, T[:4], record=True)
    Sr, r2 = O.sib_run(ref, Sr, 6, T[4:10], step0=4, record=True)
    Sr, r3 = O.midpoint_run(ref, Sr, 3, T[10:13], iters=3, step0=10, record=True)
    Sr, r4 = O.sib_run(ref, Sr, 7, T[13:], step0=13, record=True)
    assert np.abs(S - Sr).max() <= 1e-12
    rr = np.concatenate([r1, r2, r3, r4])
    assert np.abs(rec[:, 0, 7] - rr[:, 7]).max() <= 1e-12 * np.abs(rr[:, 7]).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
def test_length_kept_without_renormalisation(SS, precision, tol):
    lat = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    with SS(lat, alpha=0.1, dt=1e-15, T=300.0, S0=L.random_state(lat.n, 1), seed=5, precision=precision) as s:
        s.semi_implicit_step(500)
        S = s.spins()
    assert np.abs(np.linalg.norm(S, axis=1) - 1).max() < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_captured_steps_equal_plain_launches(SS, precision):
    lat = L.simple_cubic(10, 10, 10, J=6e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 12)
    out = {}
    for mode in ("kernels", "auto"):
        with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=6, precision=precision) as s:
            s.set_exec(mode)
            s.semi_implicit_step(70)
            s.midpoint_step(64, iterations=2)
            s.semi_implicit_step(65)
            out[mode] = (s.spins(), s.record(0, 199))
    assert np.array_equal(out["kernels"][0], out["auto"][0])
    assert np.array_equal(out["kernels"][1], out["auto"][1])


def test_invalid_arguments(SS):
    lat = L.simple_cubic(4, 4, 4, periodic=(False, False, False), with_pos=True)
    with SS(lat, T=0.0) as s:
        with pytest.raises(Exception, match=">= 0"):
            s.semi_implicit_step(-1)
        s.semi_implicit_step(2)
        assert s.step_index == 2

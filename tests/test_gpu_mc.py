"""Parity of the CUDA Monte Carlo step (through the C ABI) with the oracle.

FP64 form: the same trial moves from the same Philox blocks and the same colour order, so
the trajectories agree up to the rounding of the normalisations (held to 1e-12), the
accepted counts of every step agree exactly, and so do the records (1e-12 relative).  A
decision can only differ when dE lies within rounding of -kB T ln u, which none of these
cases comes near.  FP32-mixed form: statistical agreement (equilibrium magnetisation).
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


def _gpu_mc(SS, lat, steps, T, precision="fp64", **kw):
    with SS(lat, alpha=0.1, dt=1e-16, T=T, precision=precision, **kw) as s:
        accs, prev = [], 0
        for _ in range(steps):
            s.mc_step(1)
            a, tried = s.mc_stats(0)
            accs.append(a - prev)
            prev = a
        assert tried == steps * lat.n
        return s.spins(), s.record(0, steps), np.array(accs)


def _check_parity(S_gpu, rec_gpu, acc_gpu, S_ref, rec_ref, acc_ref):
    assert np.array_equal(acc_gpu, acc_ref)
    assert np.abs(S_gpu - S_ref).max() <= 1e-12
    g = rec_gpu[:, 0, :]
    assert np.abs(g[:, :4] - rec_ref[:, :4]).max() <= 1e-12 * np.abs(rec_ref[:, 3]).max()
    assert np.abs(g[:, 4:] - rec_ref[:, 4:]).max() <= 1e-12 * np.abs(rec_ref[:, 4:7]).max()


def test_fp64_matches_oracle_sc(SS):
    lat = L.simple_cubic(8, 8, 8, J=6.0e-21, k_u=1.0e-23)
    S0 = L.random_state(lat.n, 3)
    H = (0.0, 0.2, 0.5)
    S_gpu, rec, acc = _gpu_mc(SS, lat, 40, 400.0, S0=S0, H=H, seed=9, sys_id=2)
    S_ref, rec_ref, acc_ref = O.mc_run(oracle_system(lat, H=H, seed=9, sys_id=2), S0, 40, 400.0, record=True)
    _check_parity(S_gpu, rec, acc, S_ref, rec_ref, acc_ref)
    assert 0.1 * lat.n < acc.mean() < 0.9 * lat.n


@pytest.mark.parametrize("kind", ["fcc", "core_shell"])
def test_fp64_matches_oracle_more_colours_and_all_terms(SS, kind):
    if kind == "fcc":
        lat = L.fcc(3, 3, 3, J=11.2e-21, k_u=6.69e-24)
        T, H = 900.0, (0.3, 0.0, 0.0)
    else:
        lat = L.core_shell_sphere(diameter=3.2e-9, r_core=1.2e-9, k_s=5e-23)
        rng = np.random.default_rng(4)
        ax = rng.normal(size=(lat.n, 3))
        lat.easy_axis = ax / np.linalg.norm(ax, axis=1, keepdims=True)
        lat.k_u = rng.uniform(0, 5e-23, lat.n)
        T, H = 150.0, (0.7, -0.2, 1.0)
    S0 = L.random_state(lat.n, 11)
    S_gpu, rec, acc = _gpu_mc(SS, lat, 25, T, S0=S0, H=H, seed=77, sys_id=5)
    S_ref, rec_ref, acc_ref = O.mc_run(oracle_system(lat, H=H, seed=77, sys_id=5), S0, 25, T, record=True)
    _, nc = O.colour_greedy(oracle_system(lat))
    assert nc > 2
    _check_parity(S_gpu, rec, acc, S_ref, rec_ref, acc_ref)


def test_temperature_schedule_and_zero_temperature(SS):
    lat = L.simple_cubic(6, 6, 6, J=6.0e-21, k_u=1.0e-23)
    S0 = L.random_state(lat.n, 5)
    T = np.array([0.0, 0.0, 0.0, 50.0, 300.0, 900.0, 0.0, 0.0])
    with SS(lat, alpha=0.1, dt=1e-16, T=0.0, S0=S0, seed=4, precision="fp64") as s:
        s.set_temperature_schedule(T)
        s.mc_step(len(T))
        S_gpu = s.spins()
        rec = s.record(0, len(T))
        acc, tried = s.mc_stats(0)
    S_ref, rec_ref, acc_ref = O.mc_run(oracle_system(lat, seed=4), S0, len(T), T, record=True)
    assert acc == acc_ref.sum() and tried == lat.n * len(T)
    assert np.abs(S_gpu - S_ref).max() <= 1e-12
    E = rec[:, 0, 7]
    assert np.all(np.diff(E[:3]) <= 0)  # T = 0 steps never raise the energy
    assert np.abs(rec[:, 0, 7] - rec_ref[:, 7]).max() <= 1e-12 * np.abs(rec_ref[:, 7]).max()


def test_batch_equals_each_system_alone(SS):
    lats = [L.simple_cubic(6, 6, 6, J=6.0e-21, k_u=1e-23), L.fcc(2, 3, 2), L.simple_cubic(5, 4, 3, J=4e-21)]
    S0s = [L.random_state(l.n, 20 + k) for k, l in enumerate(lats)]
    temps = [300.0, 700.0, 0.0]
    with SS(lats, alpha=0.1, dt=1e-16, T=temps, seed=[1, 2, 3], sys_id=[0, 1, 2], S0=S0s,
            precision="fp64") as b:
        b.mc_step(12)
        S_b = b.spins()
        stats_b = [b.mc_stats(k) for k in range(3)]
    off = 0
    for k, lat in enumerate(lats):
        with SS(lat, alpha=0.1, dt=1e-16, T=temps[k], seed=k + 1, sys_id=k, S0=S0s[k], precision="fp64") as s:
            s.mc_step(12)
            assert np.array_equal(s.spins(), S_b[off:off + lat.n])
            assert s.mc_stats(0) == stats_b[k]
        off += lat.n


def test_mc_and_llg_share_the_step_counter_and_record(SS):
    lat = L.simple_cubic(6, 6, 6, J=6.0e-21, k_u=1e-23)
    with SS(lat, alpha=0.1, dt=1e-16, T=200.0, seed=6, precision="fp64") as s:
        s.mc_step(5)
        s.step(3)
        s.mc_step(2)
        assert s.step_index == 10
        rec = s.record(0, 10)
        assert np.all(np.isfinite(rec))
    ref = oracle_system(lat, seed=6)
    S, r1, _ = O.mc_run(ref, L.uniform_state(lat.n), 5, 200.0, record=True)
    S, r2 = O.heun_run(ref, S, 3, 200.0, step0=5, record=True)
    S, r3, _ = O.mc_run(ref, S, 2, 200.0, step0=8, record=True)
    rec_ref = np.concatenate([r1, r2, r3])
    assert np.abs(rec[:, 0, 7] - rec_ref[:, 7]).max() <= 1e-11 * np.abs(rec_ref[:, 7]).max()


@pytest.mark.parametrize("precision,T,tol", [("fp64", 300.0, 0.03), ("fp32", 300.0, 0.03), ("fp32", 450.0, 0.04)])
def test_equilibrium_matches_the_papers_fitted_curve(SS, precision, T, tol):
    """Fig. MCLLG's system (sc, J = 6.0e-21 J/link, periodic, 28^3): the paper's fit
    m(T) = (1 - T/Tc)^beta, Tc = 631.82 K, beta = 0.334297."""
    lat = L.simple_cubic(28, 28, 28, J=6.0e-21, k_u=0.0)
    with SS(lat, alpha=0.1, dt=1e-16, T=T, seed=31, precision=precision) as s:
        s.mc_step(400)
        first = s.step_index
        s.mc_step(400)
        rec = s.record(first, 400)
    m = np.linalg.norm(rec[:, 0, :3], axis=1) / rec[:, 0, 3]
    assert abs(m.mean() - (1 - T / 631.82) ** 0.334297) < tol


def test_fp32_mixed_boltzmann_single_spin(SS):
    """Eq. boltz through the FP32-mixed Monte Carlo: <cos^2 theta> of free spins with
    anisotropy k_u/(kB T) = 3 against the analytic distribution."""
    from scipy import integrate

    n, T, K = 20000, 50.0, 3.0
    kB = 1.3807e-23
    lat = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                        np.full(n, 1.5 * 9.274e-24), np.full(n, K * kB * T), np.tile([0.0, 0.0, 1.0], (n, 1)))
    with SS(lat, alpha=0.1, dt=1e-16, T=T, seed=3, precision="fp32") as s:
        s.mc_step(100)
        vals = []
        for _ in range(20):
            s.mc_step(5)
            vals.append(s.spins()[:, 2] ** 2)
    Z = integrate.quad(lambda x: np.exp(K * x * x), 0, 1)[0]
    ref = integrate.quad(lambda x: x * x * np.exp(K * x * x), 0, 1)[0] / Z
    assert abs(np.concatenate(vals).mean() - ref) < 0.005


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_captured_steps_equal_plain_launches(SS, precision):
    """Monte Carlo steps replayed from a captured graph (records written at the device's step)
    equal plain launches bitwise, with a temperature schedule and across graph boundaries."""
    lat = L.simple_cubic(12, 12, 12, J=6.0e-21, k_u=1e-23)
    S0 = L.random_state(lat.n, 4)
    T = np.linspace(900.0, 100.0, 150)
    out = {}
    for mode in ("kernels", "auto"):
        with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=8, precision=precision) as s:
            s.set_exec(mode)
            s.mc_step(5)
            s.set_temperature_schedule(T, step0=5)
            s.mc_step(130)
            s.step(3)
            s.mc_step(70)
            out[mode] = (s.spins(), s.record(0, 208), s.mc_stats(0))
    assert np.array_equal(out["kernels"][0], out["auto"][0])
    assert np.array_equal(out["kernels"][1], out["auto"][1])
    assert out["kernels"][2] == out["auto"][2]

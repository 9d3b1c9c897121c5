"""Deterministic (T = 0) pins of the oracle's LLG right-hand side and Heun scheme.

* Single spin in a static field against the closed form Eq. analytic_LLG, with the
  paper's printed error bound (Fig. heuntest: below 1e-6 for lambda = 0.1, H = 10 T,
  dt = 1 fs; larger for lambda = 0.05).
* Larmor period 2 pi (1 + lambda^2)/(gamma H) for an undamped spin.
* Second-order convergence: without noise Heun is a second-order Runge-Kutta scheme.
* lambda = 0: energy conservation and, for pure isotropic exchange, conservation of the
  total spin, both with an error that shrinks with dt.
* |S| = 1 after every step (renormalisation after both Heun passes).
* Stoner-Wohlfarth switching fields of a single spin at several angles (Section Test
  Simulations, angular variation of the coercivity; easy-axis coercivity H_k = 2 k_u/mu_s).
"""
import json
import os

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
GAMMA = GOLD["table_I_constants"]["gamma"]


def _single(oracle_mod, lam, H, dt, alpha_field=(0, 0, 1), mu=1.5 * L.MU_B, ku=0.0, axis=(0, 0, 1)):
    lat = L.single_spin(mu_s=mu, k_u=ku, easy_axis=axis)
    Hv = tuple(H * np.asarray(alpha_field, dtype=float))
    return oracle_mod.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis,
                                   alpha=lam, dt=dt, H_app=Hv)


def _analytic(lam, H, t):
    a = lam * GAMMA * H / (1 + lam ** 2) * t
    w = GAMMA * H / (1 + lam ** 2) * t
    return np.stack([np.cos(w) / np.cosh(a), np.sin(w) / np.cosh(a), np.tanh(a)], axis=-1)


def _trajectory_error(oracle_mod, lam, H, dt, t_end, samples=200):
    s = _single(oracle_mod, lam, H, dt)
    n = int(round(t_end / dt))
    chunk = max(1, n // samples)
    S = np.array([[1.0, 0.0, 0.0]])
    errs = []
    for k in range(n // chunk):
        S, _ = oracle_mod.heun_run(s, S, chunk, 0.0, step0=k * chunk)
        errs.append(np.abs(S[0] - _analytic(lam, H, (k + 1) * chunk * dt)).max())
    return np.array(errs)


def test_single_spin_matches_analytic_solution(oracle_mod):
    p = GOLD["single_spin_heun_test"]
    e01 = _trajectory_error(oracle_mod, p["lambda"], p["H_tesla"], p["dt_s"], 60e-12)
    assert e01.max() < p["max_error_below"], e01.max()
    assert e01.max() > 1e-8  # the characteristic Heun error trace is there, not rounding only
    e005 = _trajectory_error(oracle_mod, 0.05, p["H_tesla"], p["dt_s"], 60e-12)
    assert e005.max() > 1.5 * e01.max()  # lower damping -> larger error (Fig. heuntest b, d)


def test_larmor_period(oracle_mod):
    H, dt = 10.0, 1e-16
    s = _single(oracle_mod, 0.0, H, dt)
    period = 2 * np.pi / (GAMMA * H)
    assert abs(period - 3.570e-12) < 1e-15
    nsteps = int(round(period / dt))
    S, _ = oracle_mod.heun_run(s, np.array([[1.0, 0, 0]]), nsteps, 0.0)
    # back to the start after one period, up to the sub-step remainder
    rem = period - nsteps * dt
    phase = GAMMA * H * (nsteps * dt)
    np.testing.assert_allclose(S[0], [np.cos(phase), np.sin(phase), 0.0], atol=1e-7)
    assert abs(rem) < dt
    # damping slows precession by (1 + lambda^2)
    lam = 0.5
    s = _single(oracle_mod, lam, H, dt)
    t = 1e-12
    S, _ = oracle_mod.heun_run(s, np.array([[1.0, 0, 0]]), int(round(t / dt)), 0.0)
    np.testing.assert_allclose(S[0], _analytic(lam, H, t), atol=1e-7)


def test_second_order_convergence(oracle_mod):
    errs = [_trajectory_error(oracle_mod, 0.1, 10.0, dt, 20e-12, samples=50).max() for dt in (4e-15, 2e-15, 1e-15)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


def _lattice_system(oracle_mod, lat, lam, dt, H=(0, 0, 0), ku=None):
    return oracle_mod.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u if ku is None else ku,
                                   lat.easy_axis, alpha=lam, dt=dt, H_app=H)


def test_undamped_energy_conservation(oracle_mod):
    lat = L.simple_cubic(4, 4, 4, k_u=2e-22)
    S0 = L.random_state(lat.n, 21)
    drifts = []
    for dt in (4e-17, 2e-17):
        s = _lattice_system(oracle_mod, lat, 0.0, dt, H=(0.3, 0.0, 5.0))
        e0 = oracle_mod.moment_energy(s, S0)[7]
        S, _ = oracle_mod.heun_run(s, S0, int(round(2e-13 / dt)), 0.0)
        drifts.append(abs(oracle_mod.moment_energy(s, S)[7] - e0) / abs(e0))
    assert drifts[0] < 1e-3
    assert drifts[0] / drifts[1] > 3.0, drifts  # second order in dt


def test_undamped_isotropic_exchange_conserves_total_spin(oracle_mod):
    lat = L.simple_cubic(4, 4, 4, k_u=0.0)
    S0 = L.random_state(lat.n, 22)
    drifts = []
    for dt in (4e-17, 2e-17):
        s = _lattice_system(oracle_mod, lat, 0.0, dt)
        S, _ = oracle_mod.heun_run(s, S0, int(round(2e-13 / dt)), 0.0)
        drifts.append(np.abs(S.sum(0) - S0.sum(0)).max() / lat.n)
    assert drifts[0] < 1e-4
    assert drifts[0] / drifts[1] > 3.0, drifts


def test_unit_length_after_every_step(oracle_mod):
    lat = L.simple_cubic(5, 5, 5)
    s = _lattice_system(oracle_mod, lat, 0.1, 1e-16)
    S = L.random_state(lat.n, 3)
    for k in range(20):
        S, _ = oracle_mod.heun_run(s, S, 1, 900.0, step0=k)
        np.testing.assert_allclose(np.linalg.norm(S, axis=1), 1.0, atol=4e-16)


def _sw_switching_field(psi):
    """Stoner-Wohlfarth astroid: h_sw = (cos^(2/3) psi + sin^(2/3) psi)^(-3/2)."""
    c, s = abs(np.cos(psi)), abs(np.sin(psi))
    return (c ** (2 / 3) + s ** (2 / 3)) ** -1.5


def test_stoner_wohlfarth_switching(oracle_mod):
    p = GOLD["stoner_wohlfarth_test"]
    ku, mu = 1e-22, 1.5 * L.MU_B
    Hk = 2 * ku / mu
    psis = np.deg2rad([0.01, 20.0, 45.0, 70.0])
    lat = L.single_spin(mu_s=mu, k_u=ku)
    n = len(psis)
    # independent spins with easy axes at angle psi from the field (+z), in the xz plane
    axes = np.stack([np.sin(psis), np.zeros(n), np.cos(psis)], 1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    dt = 0.01 / (GAMMA * Hk)
    S = np.tile([0.0, 0.0, 1.0], (n, 1))
    switched_at = np.full(n, np.nan)
    h = 1.2
    while h > -1.2:
        s = oracle_mod.OracleSystem(row_ptr, lat.col, lat.J, np.full(n, mu), np.full(n, ku), axes,
                                    alpha=1.0, dt=dt, H_app=(0.0, 0.0, h * Hk))
        S_before = S.copy()
        for _ in range(400):
            S, _ = oracle_mod.heun_run(s, S, 200, 0.0)
            torque = np.linalg.norm(np.cross(S, oracle_mod.fields(s, S)), axis=1)
            if torque.max() <= p["torque_tolerance_tesla"]:
                break
        # an irreversible jump between neighbouring field steps marks the switching field
        jump = np.linalg.norm(S - S_before, axis=1) > 0.3
        newly = np.isnan(switched_at) & jump & (h < 0)
        switched_at[newly] = h
        h = round(h - p["field_step_over_Hk"], 10)
    expect = np.array([_sw_switching_field(x) for x in psis])
    # the spin jumps at the first field step at or beyond -h_sw
    assert np.all(np.abs(-switched_at - expect) <= p["field_step_over_Hk"] + 1e-9), (switched_at, expect)
    # easy-axis coercivity is H_k = 2 k_u / mu_s itself (0.01 degrees off axis: h_sw = 0.995)
    assert abs(-switched_at[0] - 1.0) <= p["field_step_over_Hk"] + 1e-9

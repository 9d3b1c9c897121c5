"""Pins of the oracle's midpoint integrator (the midpoint rule the paper's time-integration
section cites as the alternative to Heun; readings I1-I3).

  * the rule keeps |S| without renormalisation: the length error after 100 steps of a
    300 K lattice falls geometrically with the number of fixed-point iterations K;
  * undamped precession of a single spin in a static field: the converged midpoint rule is
    the Cayley rotation, advancing the azimuth by exactly 2 atan(w dt / 2) per step, with S_z
    and |S| conserved;
  * the damped single spin against the closed form Eq. analytic_LLG converges at second
    order (halving dt divides the error by ~4);
  * the Boltzmann distribution of a single spin with anisotropy (Eq. boltz) with the thermal
    field held over each step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

GAMMA, KB, MU = 1.76e11, 1.3807e-23, 1.5 * 9.2740e-24


def _single(lam, H, dt, ku=0.0):
    return O.OracleSystem(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), [MU], ku, (0, 0, 1),
                          alpha=lam, dt=dt, H_app=(0.0, 0.0, H), seed=3)


def test_length_error_falls_geometrically_with_iterations():
    lat = L.simple_cubic(5, 5, 5, J=6e-21, k_u=1e-23)
    s = oracle_system(lat, alpha=0.1, dt=1e-16, seed=2)
    S0 = L.random_state(lat.n, 1)
    errs = []
    for K in (2, 4, 8, 12):
        S, _ = O.midpoint_run(s, S0, 100, 300.0, iters=K)
        errs.append(np.abs(np.linalg.norm(S, axis=1) - 1).max())
    assert errs[-1] < 1e-13
    assert errs[0] > 100 * errs[1] > 100 * 100 * errs[2]


def test_undamped_precession_is_the_cayley_rotation():
    H = 10.0
    w = GAMMA * H
    dt = 0.1 / w
    s = _single(0.0, H, dt)
    S0 = np.array([[0.6, 0.0, 0.8]])
    S, _ = O.midpoint_run(s, S0, 100, 0.0, iters=40)
    phi = np.arctan2(S[0, 1], S[0, 0])
    # dS/dt = -gamma S x H with H along +z turns S anticlockwise; the midpoint rule by 2 atan(w dt/2) a step
    expected = np.angle(np.exp(1j * 100 * 2 * np.arctan(w * dt / 2)))
    assert abs(np.angle(np.exp(1j * (phi - expected)))) < 1e-10
    assert S[0, 2] == pytest.approx(0.8, abs=1e-14)
    assert np.linalg.norm(S[0]) == pytest.approx(1.0, abs=1e-14)


def _analytic(lam, H, t):
    a = lam * GAMMA * H / (1 + lam ** 2) * t
    w = GAMMA * H / (1 + lam ** 2) * t
    return np.array([np.cos(w) / np.cosh(a), np.sin(w) / np.cosh(a), np.tanh(a)])


def test_damped_single_spin_converges_at_second_order():
    lam, H, t_end = 0.1, 10.0, 20e-12
    errs = []
    for dt in (4e-15, 2e-15, 1e-15):
        n = int(round(t_end / dt))
        S, _ = O.midpoint_run(_single(lam, H, dt), np.array([[1.0, 0.0, 0.0]]), n, 0.0, iters=30)
        ref = _analytic(lam, H, t_end)
        errs.append(np.abs(S[0] - ref).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
    assert errs[2] < 1e-3


def test_boltzmann_distribution_with_the_midpoint_rule():
    from scipy import integrate

    ku, kappa, lam = 1e-22, 3.0, 1.0
    T = ku / (kappa * KB)
    dt = 0.005 * MU / (2 * lam * KB * T * GAMMA)
    n = 200
    s = O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, MU), ku,
                       (0, 0, 1), alpha=lam, dt=dt, seed=5)
    O.set_threads(O.max_threads())
    try:
        S, _ = O.midpoint_run(s, np.tile([0, 0, 1.0], (n, 1)), 2000, T, iters=6)
        c2 = []
        for k in range(60):
            S, _ = O.midpoint_run(s, S, 300, T, iters=6, step0=2000 + 300 * k)
            c2.append(S[:, 2] ** 2)
    finally:
        O.set_threads(1)
    Z = integrate.quad(lambda x: np.exp(kappa * x * x), 0, 1)[0]
    ref = integrate.quad(lambda x: x * x * np.exp(kappa * x * x), 0, 1)[0] / Z
    assert abs(np.concatenate(c2).mean() - ref) < 0.015

"""Pins of the oracle's semi-implicit predictor-corrector (the modified predictor-corrector
midpoint scheme the paper cites, Mentink et al. 2010, scheme B; readings P1-P3).

  * a single spin with anisotropy and an oblique field against the scheme's two defining
    linear equations solved independently (numpy's dense solver) step by step;
  * undamped precession in a static field: both half-steps are the Cayley rotation, so the
    azimuth advances by exactly 2 atan(w dt / 2) per step with S_z and |S| conserved;
  * |S| is kept without renormalisation on a 300 K lattice with a large time step;
  * the damped single spin against the closed form Eq. analytic_LLG converges at second order;
  * the Boltzmann distribution of a single spin with anisotropy (Eq. boltz): the scheme
    reaches the Stratonovich equilibrium with the thermal field held over each step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

GAMMA, KB, MU = 1.76e11, 1.3807e-23, 1.5 * 9.2740e-24


def _single(lam, H, dt, ku=0.0, axis=(0, 0, 1)):
    return O.OracleSystem(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), [MU], ku, axis,
                          alpha=lam, dt=dt, H_app=tuple(H) if np.ndim(H) else (0.0, 0.0, H), seed=3)


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])  # _skew(v) @ x = v x x


def test_single_spin_against_the_defining_equations():
    lam, ku, dt = 0.3, 2e-23, 2e-15
    e = np.array([0.3, -0.2, 0.9])
    e /= np.linalg.norm(e)
    Happ = np.array([0.4, 1.1, -0.7])
    s = _single(lam, Happ, dt, ku=ku, axis=tuple(e))
    S = np.array([0.48, 0.6, 0.64])

    def A(v):  # -gamma/(1+lam^2) (H + lam v x H), H the field at v
        H = Happ + 2 * ku / MU * (v @ e) * e
        return -GAMMA / (1 + lam ** 2) * (H + lam * np.cross(v, H))

    def half(Sn, a):  # X = Sn + (dt/2)(Sn + X) x a  <=>  (I - (dt/2) [.] x a) X = Sn + (dt/2) Sn x a
        M = np.eye(3) + (dt / 2) * _skew(a)  # (Sn + X) x a = -a x (Sn + X)
        return np.linalg.solve(M, Sn - (dt / 2) * np.cross(a, Sn))

    ref = S.copy()
    for _ in range(20):
        P = half(ref, A(ref))
        ref = half(ref, A(0.5 * (ref + P)))
    got, _ = O.sib_run(s, S[None], 20, 0.0)
    assert np.abs(got[0] - ref).max() <= 1e-13


def test_undamped_precession_is_the_cayley_rotation():
    H = 10.0
    w = GAMMA * H
    dt = 0.1 / w
    S, _ = O.sib_run(_single(0.0, H, dt), np.array([[0.6, 0.0, 0.8]]), 100, 0.0)
    phi = np.arctan2(S[0, 1], S[0, 0])
    expected = np.angle(np.exp(1j * 100 * 2 * np.arctan(w * dt / 2)))
    assert abs(np.angle(np.exp(1j * (phi - expected)))) < 1e-10
    assert S[0, 2] == pytest.approx(0.8, abs=1e-14)
    assert np.linalg.norm(S[0]) == pytest.approx(1.0, abs=1e-14)


def test_length_kept_without_renormalisation():
    lat = L.simple_cubic(5, 5, 5, J=6e-21, k_u=1e-23)
    S, _ = O.sib_run(oracle_system(lat, alpha=0.1, dt=1e-15, seed=2), L.random_state(lat.n, 1), 500, 300.0)
    assert np.abs(np.linalg.norm(S, axis=1) - 1).max() < 1e-13


def _analytic(lam, H, t):
    a = lam * GAMMA * H / (1 + lam ** 2) * t
    w = GAMMA * H / (1 + lam ** 2) * t
    return np.array([np.cos(w) / np.cosh(a), np.sin(w) / np.cosh(a), np.tanh(a)])


def test_damped_single_spin_converges_at_second_order():
    lam, H, t_end = 0.1, 10.0, 20e-12
    errs = []
    for dt in (4e-15, 2e-15, 1e-15):
        S, _ = O.sib_run(_single(lam, H, dt), np.array([[1.0, 0.0, 0.0]]), int(round(t_end / dt)), 0.0)
        errs.append(np.abs(S[0] - _analytic(lam, H, t_end)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
    assert errs[2] < 1e-6


def test_boltzmann_distribution():
    from scipy import integrate

    ku, kappa, lam = 1e-22, 3.0, 1.0
    T = ku / (kappa * KB)
    dt = 0.005 * MU / (2 * lam * KB * T * GAMMA)
    n = 200
    s = O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, MU), ku,
                       (0, 0, 1), alpha=lam, dt=dt, seed=5)
    O.set_threads(O.max_threads())
    try:
        S, _ = O.sib_run(s, np.tile([0, 0, 1.0], (n, 1)), 2000, T)
        c2 = []
        for k in range(60):
            S, _ = O.sib_run(s, S, 300, T, step0=2000 + 300 * k)
            c2.append(S[:, 2] ** 2)
    finally:
        O.set_threads(1)
    Z = integrate.quad(lambda x: np.exp(kappa * x * x), 0, 1)[0]
    ref = integrate.quad(lambda x: x * x * np.exp(kappa * x * x), 0, 1)[0] / Z
    assert abs(np.concatenate(c2).mean() - ref) < 0.015

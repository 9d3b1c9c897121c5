"""Pins of the oracle's tensorial exchange (Eqs. HJijM, HJijSMS) and cubic anisotropy.

  * the energy against a brute-force sum of the printed expressions: -S_i . J_ij S_j over the
    bonds (each once) and (k_c/2)(Sx^4 + Sy^4 + Sz^4) per atom;
  * the field against -(1/mu_s) dE/dS by central differences of that brute-force energy, with
    random tensors (a symmetric two-ion part and an antisymmetric Dzyaloshinskii-Moriya part)
    whose reverse bonds carry the transpose, and random k_c;
  * a scalar J written as J times the identity tensor gives the scalar trajectory bitwise;
  * a Heisenberg + DM dimer relaxes (LLG at T = 0) to the closed-form ground state: S1 and S2
    perpendicular to D at the angle with tan = |D|/J, the chirality S1 x S2 antiparallel to D for
    E = -J S1.S2 + D.(S1 x S2), and E = -sqrt(J^2 + |D|^2); Monte Carlo at 1 K sits there too;
  * a single spin with cubic anisotropy relaxes to <100> for k_c < 0 and to <111> for k_c > 0,
    and the energies of [100], [110], [111] are k_c/2, k_c/4, k_c/6;
  * Monte Carlo of free spins with cubic anisotropy reproduces the Boltzmann average of
    Sx^4 + Sy^4 + Sz^4 over the sphere.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_1310_6143_gb300 import lattice as L

MU_B = 9.2740e-24
KB = 1.3807e-23


def _skew(d):
    return np.array([[0.0, -d[2], d[1]], [d[2], 0.0, -d[0]], [-d[1], d[0], 0.0]])  # _skew(d) @ x = d x x


def _tensor_system(lat, rng, scale=6e-21):
    """Random bond tensors with J_ji = J_ij^T: J * I + symmetric two-ion part + DM part."""
    n = lat.n
    rows = np.repeat(np.arange(n), np.diff(lat.row_ptr))
    Jt = np.zeros((lat.nnz, 3, 3))
    where = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(rows, lat.col))}
    for k, (i, j) in enumerate(zip(rows, lat.col)):
        if i < j:
            B = rng.normal(size=(3, 3)) * 0.2 * scale
            A = scale * np.eye(3) + 0.5 * (B + B.T) + _skew(rng.normal(size=3) * 0.3 * scale)
            Jt[k] = A
            Jt[where[(int(j), int(i))]] = A.T
    mu = np.full(n, 1.5 * MU_B) * rng.uniform(0.8, 1.2, n)
    kc = rng.uniform(-2e-23, 2e-23, n)
    s = O.OracleSystem(lat.row_ptr, lat.col, np.zeros(lat.nnz), mu, 1e-23, (0, 0, 1), J_tensor=Jt, k_c=kc,
                       H_app=(0.1, -0.2, 0.3))
    return s, Jt, mu, kc, rows


def _brute(S, s, Jt, mu, kc, rows):
    eex = 0.0
    for k, (i, j) in enumerate(zip(rows, s.col)):
        if i < j:
            eex -= S[i] @ Jt[k] @ S[j]
    ean = -np.sum(1e-23 * S[:, 2] ** 2) + np.sum(0.5 * kc * (S ** 4).sum(1))
    eap = -np.sum(mu * (S @ np.array(s.H_app)))
    return eex, ean, eap


def test_energy_matches_bruteforce_with_tensors_and_cubic():
    lat = L.simple_cubic(3, 3, 3)
    s, Jt, mu, kc, rows = _tensor_system(lat, np.random.default_rng(1))
    S = L.random_state(lat.n, 3)
    out = O.moment_energy(s, S)
    np.testing.assert_allclose(out[4:7], _brute(S, s, Jt, mu, kc, rows), rtol=1e-12, atol=1e-36)


def test_field_is_energy_gradient_with_tensors_and_cubic():
    lat = L.simple_cubic(3, 3, 3)
    s, Jt, mu, kc, rows = _tensor_system(lat, np.random.default_rng(2))
    S = L.random_state(lat.n, 4)
    Hf = O.fields(s, S)
    h = 1e-6
    for i in range(lat.n):
        for c in range(3):
            Sp = S.copy(); Sp[i, c] += h
            Sm = S.copy(); Sm[i, c] -= h
            dE = (sum(_brute(Sp, s, Jt, mu, kc, rows)) - sum(_brute(Sm, s, Jt, mu, kc, rows))) / (2 * h)
            assert abs(Hf[i, c] + dE / mu[i]) <= 1e-7 * max(1.0, np.abs(Hf[i]).max()), (i, c)


def test_identity_tensor_equals_scalar_exchange():
    lat = L.simple_cubic(5, 5, 5, J=6e-21, k_u=1e-23)
    a = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, seed=3)
    b = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, seed=3,
                       J_tensor=lat.J[:, None, None] * np.eye(3)[None])
    S0 = L.random_state(lat.n, 5)
    Sa, ra = O.heun_run(a, S0, 30, 300.0, record=True)
    Sb, rb = O.heun_run(b, S0, 30, 300.0, record=True)
    assert np.array_equal(Sa, Sb) and np.array_equal(ra, rb)


def _dm_dimer(J, D):
    A = J * np.eye(3) + _skew(D)
    return O.OracleSystem(np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32), np.zeros(2), np.full(2, 2 * MU_B),
                          0.0, (0, 0, 1), J_tensor=np.stack([A, A.T]), alpha=1.0, dt=1e-16, seed=4)


def test_dm_dimer_relaxes_to_the_closed_form_ground_state():
    J, D = 5e-21, np.array([1.0, -2.0, 2.0]) * 1e-21  # |D| = 3e-21
    s = _dm_dimer(J, D)
    S, _ = O.heun_run(s, L.random_state(2, 6), 40000, 0.0)
    Dn = np.linalg.norm(D)
    E = O.moment_energy(s, S)[7]
    assert E == pytest.approx(-np.hypot(J, Dn), rel=1e-6, abs=0)
    assert S[0] @ S[1] == pytest.approx(J / np.hypot(J, Dn), abs=1e-4)
    assert np.cross(S[0], S[1]) @ (D / Dn) == pytest.approx(-Dn / np.hypot(J, Dn), abs=1e-4)
    assert abs(S[0] @ D) < 1e-3 * Dn and abs(S[1] @ D) < 1e-3 * Dn


def test_dm_dimer_monte_carlo_near_the_ground_state():
    """At 1 K (kB T ~ 0.2 % of the bond energy) the Monte Carlo dimer sits at the closed-form
    ground state up to thermal fluctuations, with its chirality."""
    J, D = 5e-21, np.array([1.0, -2.0, 2.0]) * 1e-21
    s = _dm_dimer(J, D)
    S, _, _ = O.mc_run(s, L.random_state(2, 6), 3000, 1.0)
    _, rec, _ = O.mc_run(s, S, 2000, 1.0, step0=3000, record=True)
    Dn = np.linalg.norm(D)
    assert rec[:, 7].mean() == pytest.approx(-np.hypot(J, Dn), rel=0.01, abs=0)
    S, _, _ = O.mc_run(s, S, 1, 1.0, step0=5000)
    assert np.cross(S[0], S[1]) @ (D / Dn) == pytest.approx(-Dn / np.hypot(J, Dn), abs=0.08)


def test_cubic_anisotropy_energies_and_easy_axes():
    kc = 3e-23
    one = dict(row_ptr=np.array([0, 0]), col=np.zeros(0, dtype=np.int32), J=np.zeros(0), mu_s=[2 * MU_B], k_u=0.0,
               easy_axis=(0, 0, 1))
    s = O.OracleSystem(**one, k_c=kc)
    for d, e in (([1, 0, 0], kc / 2), ([1, 1, 0], kc / 4), ([1, 1, 1], kc / 6)):
        v = np.array(d, dtype=float) / np.linalg.norm(d)
        assert O.moment_energy(s, v[None])[5] == pytest.approx(e, rel=1e-14, abs=0)
    start = np.array([[0.3, 0.5, 0.81]])
    start /= np.linalg.norm(start)
    for sign, target in ((1.0, np.ones(3) / np.sqrt(3)), (-1.0, np.array([0, 0, 1.0]))):
        sr = O.OracleSystem(**one, k_c=sign * 2e-22, alpha=1.0, dt=1e-15, seed=1)  # 60 ps at 2k_c/mu = 22 T
        S, _ = O.heun_run(sr, start, 60000, 0.0)
        assert np.abs(np.abs(S[0]) - target).max() < 1e-4


def test_monte_carlo_cubic_boltzmann_average():
    n, T, K = 4000, 40.0, 4.0  # k_c/(kB T)
    kc = K * KB * T
    s = O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                       np.full(n, 2 * MU_B), 0.0, (0, 0, 1), k_c=kc, seed=12)
    S, _, _ = O.mc_run(s, L.random_state(n, 1), 80, T)
    vals, step = [], 80
    for _ in range(20):
        S, _, _ = O.mc_run(s, S, 5, T, step0=step)
        step += 5
        vals.append((S ** 4).sum(1))
    f = lambda th, ph: (np.sin(th) ** 4 * (np.cos(ph) ** 4 + np.sin(ph) ** 4) + np.cos(th) ** 4)  # noqa: E731
    w = lambda th, ph: np.exp(-0.5 * K * f(th, ph)) * np.sin(th)  # noqa: E731
    Z = integrate.dblquad(lambda th, ph: w(th, ph), 0, 2 * np.pi, 0, np.pi)[0]
    ref = integrate.dblquad(lambda th, ph: f(th, ph) * w(th, ph), 0, 2 * np.pi, 0, np.pi)[0] / Z
    assert np.concatenate(vals).mean() == pytest.approx(ref, abs=0.004)

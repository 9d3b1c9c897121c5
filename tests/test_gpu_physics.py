"""Closed-form physics checks of the CUDA path itself (the oracle's dynamics and statistics pins,
run through the C ABI): the Larmor period, second-order convergence of Heun at T = 0 to the
closed form Eq. analytic_LLG, energy and total-spin conservation without damping, Stoner-
Wohlfarth switching (angular variation of the coercivity, easy-axis coercivity 2 k_u/mu_s), the
Langevin function <cos theta> = coth x - 1/x and the Boltzmann distribution (Eq. boltz) reached by
the stochastic LLG at finite T, and the LLG equilibrium magnetisation of the paper's sc 28^3
system against its fitted m(T) (Fig. MCLLG)."""
import json
import os

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
GAMMA = GOLD["table_I_constants"]["gamma"]
KB = 1.3807e-23


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _analytic(lam, H, t):
    a = lam * GAMMA * H / (1 + lam ** 2) * t
    w = GAMMA * H / (1 + lam ** 2) * t
    return np.array([np.cos(w) / np.cosh(a), np.sin(w) / np.cosh(a), np.tanh(a)])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-7), ("fp32", 2e-4)])
def test_larmor_period(SS, precision, tol):
    H, dt = 10.0, 1e-16
    period = 2 * np.pi / (GAMMA * H)
    n = int(round(period / dt))
    with SS(L.single_spin(), alpha=0.0, dt=dt, T=0.0, H=(0.0, 0.0, H), S0=np.array([[1.0, 0.0, 0.0]]),
            precision=precision) as s:
        s.step(n)
        S = s.spins()[0]
    phase = GAMMA * H * n * dt
    np.testing.assert_allclose(S, [np.cos(phase), np.sin(phase), 0.0], atol=tol)


def test_heun_second_order_convergence(SS):
    lam, H, t_end = 0.1, 10.0, 20e-12
    errs = []
    for dt in (4e-15, 2e-15, 1e-15):
        with SS(L.single_spin(), alpha=lam, dt=dt, T=0.0, H=(0.0, 0.0, H), S0=np.array([[1.0, 0.0, 0.0]]),
                precision="fp64") as s:
            s.step(int(round(t_end / dt)))
            errs.append(np.abs(s.spins()[0] - _analytic(lam, H, t_end)).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs
    assert errs[1] < GOLD["single_spin_heun_test"]["max_error_below"] * 4  # dt = 2 fs: 4x the 1 fs bound


def test_undamped_energy_and_total_spin_conservation(SS):
    lat = L.simple_cubic(4, 4, 4, k_u=2e-22)
    S0 = L.random_state(lat.n, 21)
    drifts = []
    for dt in (4e-17, 2e-17):
        with SS(lat, alpha=0.0, dt=dt, T=0.0, H=(0.3, 0.0, 5.0), S0=S0, precision="fp64") as s:
            e0 = s.energy()[0]
            s.step(int(round(2e-13 / dt)))
            drifts.append(abs(s.energy()[0] - e0) / abs(e0))
    assert drifts[0] < 1e-3 and drifts[0] / drifts[1] > 3.0, drifts
    iso = L.simple_cubic(4, 4, 4, k_u=0.0)
    S0 = L.random_state(iso.n, 22)
    drifts = []
    for dt in (4e-17, 2e-17):
        with SS(iso, alpha=0.0, dt=dt, T=0.0, S0=S0, precision="fp64") as s:
            s.step(int(round(2e-13 / dt)))
            drifts.append(np.abs(s.spins().sum(0) - S0.sum(0)).max() / iso.n)
    assert drifts[0] < 1e-4 and drifts[0] / drifts[1] > 3.0, drifts


def _sw_switching_field(psi):
    """Stoner-Wohlfarth astroid: h_sw = (cos^(2/3) psi + sin^(2/3) psi)^(-3/2)."""
    c, s = abs(np.cos(psi)), abs(np.sin(psi))
    return (c ** (2 / 3) + s ** (2 / 3)) ** -1.5


def test_stoner_wohlfarth_switching(SS):
    p = GOLD["stoner_wohlfarth_test"]
    ku, mu = 1e-22, 1.5 * L.MU_B
    Hk = 2 * ku / mu
    psis = np.deg2rad([0.01, 20.0, 45.0, 70.0])
    n = len(psis)
    axes = np.stack([np.sin(psis), np.zeros(n), np.cos(psis)], 1)  # easy axes at psi from the field (+z)
    lat = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, mu),
                        np.full(n, ku), axes)
    dt = 0.01 / (GAMMA * Hk)
    switched_at = np.full(n, np.nan)
    with SS(lat, alpha=1.0, dt=dt, T=0.0, S0=np.tile([0.0, 0.0, 1.0], (n, 1)), precision="fp64") as s:
        S = s.spins()
        h = 1.2
        while h > -1.2:
            s.set_field((0.0, 0.0, h * Hk))
            S_before = S.copy()
            for _ in range(400):
                s.step(200)
                S = s.spins()
                Hf = np.array([0.0, 0.0, h * Hk]) + (2 * ku / mu) * (S * axes).sum(1)[:, None] * axes
                if np.linalg.norm(np.cross(S, Hf), axis=1).max() <= p["torque_tolerance_tesla"]:
                    break
            jump = np.linalg.norm(S - S_before, axis=1) > 0.3
            switched_at[np.isnan(switched_at) & jump & (h < 0)] = h
            h = round(h - p["field_step_over_Hk"], 10)
    expect = np.array([_sw_switching_field(x) for x in psis])
    assert np.all(np.abs(-switched_at - expect) <= p["field_step_over_Hk"] + 1e-9), (switched_at, expect)
    assert abs(-switched_at[0] - 1.0) <= p["field_step_over_Hk"] + 1e-9  # easy-axis coercivity H_k


def _langevin(x):
    return 1.0 / np.tanh(x) - 1.0 / x


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_langevin_function_from_the_stochastic_llg(SS, precision):
    """Free spins (no exchange, no anisotropy) in a field at temperature T: the stochastic
    LLG with the Heun step reaches <cos theta> = L(mu_s H / kB T) (the Stratonovich limit)."""
    n, T, x, lam = 20000, 50.0, 2.0, 1.0
    mu = 1.5 * L.MU_B
    H = x * KB * T / mu
    dt = 0.005 * mu / (2 * lam * KB * T * GAMMA)
    lat = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, mu),
                        np.zeros(n), np.tile([0.0, 0.0, 1.0], (n, 1)))
    with SS(lat, alpha=lam, dt=dt, T=T, H=(0.0, 0.0, H), seed=17, precision=precision) as s:
        s.step(2000)
        c = []
        for _ in range(60):
            s.step(300)
            c.append(s.spins()[:, 2])
    assert abs(np.concatenate(c).mean() - _langevin(x)) < 0.01


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_boltzmann_distribution_from_the_stochastic_llg(SS, precision):
    """Eq. boltz: free spins with uniaxial anisotropy, k_u/(kB T) = 3, sample cos theta with
    density proportional to exp(3 cos^2 theta); the histogram of 20 bins matches it."""
    n, kappa, lam = 20000, 3.0, 1.0
    mu = 1.5 * L.MU_B
    ku = 1e-22
    T = ku / (kappa * KB)
    dt = 0.005 * mu / (2 * lam * KB * T * GAMMA)
    lat = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, mu),
                        np.full(n, ku), np.tile([0.0, 0.0, 1.0], (n, 1)))
    with SS(lat, alpha=lam, dt=dt, T=T, seed=23, precision=precision) as s:
        s.step(2000)
        c = []
        for _ in range(60):
            s.step(300)
            c.append(s.spins()[:, 2])
    c = np.concatenate(c)
    edges = np.linspace(-1.0, 1.0, 21)
    hist = np.histogram(c, bins=edges)[0] / c.size
    from scipy import integrate

    Z = integrate.quad(lambda u: np.exp(kappa * u * u), -1, 1)[0]
    expect = np.array([integrate.quad(lambda u: np.exp(kappa * u * u), a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    expect /= Z
    assert np.abs(hist - expect).max() < 0.006, np.abs(hist - expect).max()


@pytest.mark.parametrize("precision,T,tol", [("fp64", 300.0, 0.03), ("fp32", 450.0, 0.04)])
def test_llg_equilibrium_matches_the_papers_fitted_curve(SS, precision, T, tol):
    """Fig. MCLLG: the LLG equilibrium magnetisation of the sc 28^3 system (J = 6.0e-21 J/link,
    periodic) follows the paper's fit m(T) = (1 - T/Tc)^beta, Tc = 631.82 K, beta = 0.334297, as
    its Monte Carlo does."""
    lat = L.simple_cubic(28, 28, 28, J=6.0e-21, k_u=0.0)
    with SS(lat, alpha=1.0, dt=5e-16, T=T, seed=41, precision=precision) as s:
        s.step(6000)
        first = s.step_index
        s.step(4000)
        rec = s.record(first, 4000)
    m = np.linalg.norm(rec[:, 0, :3], axis=1) / rec[:, 0, 3]
    assert abs(m.mean() - (1 - T / 631.82) ** 0.334297) < tol

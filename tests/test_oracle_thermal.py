"""Thermal (Langevin) pins of the oracle.

* Boltzmann distribution of a single spin with uniaxial anisotropy, reflected about
  pi/2 (Section Test Simulations, Eq. boltz): with c = |cos theta|,
  P(c) ~ exp(k_u c^2 / (k_B T)) on [0, 1].  Checked by a Kolmogorov-Smirnov test and by
  <c^2>; a factor-2 error in the noise variance moves <c^2> by ~30 standard errors.
* Langevin function: a free spin in a field has <cos theta> = coth x - 1/x,
  x = mu_s H / (k_B T) (Boltzmann statistics of the Zeeman term).
* Curie temperature: the simple-cubic ferromagnet with J = 6.0e-21 J/link orders below
  and is disordered above the Tc ~ 625 K that Eq. JijTc gives (Fig. MCLLG caption); a
  double-counted (or halved) exchange field would move Tc by a factor two.
"""
import json
import os

import numpy as np
from scipy import integrate, stats

from paper_1310_6143_gb300 import lattice as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
KB = GOLD["table_I_constants"]["k_B"]
GAMMA = GOLD["table_I_constants"]["gamma"]
MU = 1.5 * GOLD["table_I_constants"]["mu_B"]


def _free_spins(oracle_mod, n, ku, lam, dt, H=(0, 0, 0), seed=5):
    return oracle_mod.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0),
                                   np.full(n, MU), np.full(n, ku), (0, 0, 1), alpha=lam, dt=dt, H_app=H,
                                   seed=seed)


def test_single_spin_boltzmann_distribution(oracle_mod):
    ku, kappa, lam = 1e-22, 3.0, 1.0
    T = ku / (kappa * KB)
    # step chosen so the rms thermal kick per step is 0.05 rad
    dt = 0.0025 * MU / (2 * lam * KB * T * GAMMA)
    n = 64
    s = _free_spins(oracle_mod, n, ku, lam, dt)
    S, _ = oracle_mod.heun_run(s, np.tile([0, 0, 1.0], (n, 1)), 5000, T)
    thin, samples = 400, []
    for k in range(300):
        S, _ = oracle_mod.heun_run(s, S, thin, T, step0=5000 + k * thin)
        samples.append(np.abs(S[:, 2]))
    c = np.concatenate(samples)
    Z = integrate.quad(lambda x: np.exp(kappa * x * x), 0, 1)[0]

    def cdf(v):
        return np.array([integrate.quad(lambda y: np.exp(kappa * y * y), 0, x)[0] / Z for x in np.atleast_1d(v)])

    assert stats.kstest(c, cdf).pvalue > 1e-3
    m2 = integrate.quad(lambda x: x * x * np.exp(kappa * x * x), 0, 1)[0] / Z
    se = (c * c).std() / np.sqrt(c.size)
    assert abs((c * c).mean() - m2) < 4 * se + 2e-3, ((c * c).mean(), m2, se)


def test_langevin_function(oracle_mod):
    T, x, lam = 300.0, 3.0, 1.0
    H = x * KB * T / MU
    dt = 0.0025 * MU / (2 * lam * KB * T * GAMMA)
    n = 128
    s = _free_spins(oracle_mod, n, 0.0, lam, dt, H=(0, 0, H), seed=6)
    S, _ = oracle_mod.heun_run(s, np.tile([0, 0, 1.0], (n, 1)), 3000, T)
    S, rec = oracle_mod.heun_run(s, S, 60000, T, step0=3000, record=True)
    m = rec[:, 2] / rec[:, 3]
    batches = m.reshape(30, -1).mean(1)
    se = batches.std(ddof=1) / np.sqrt(batches.size)
    expect = 1 / np.tanh(x) - 1 / x
    assert abs(m.mean() - expect) < 4 * se + 2e-3, (m.mean(), expect, se)


def test_magnetisation_vanishes_above_tc(oracle_mod):
    p = GOLD["curie_sc_llg"]
    Tc = p["Tc_from_eq_JijTc"]
    lat = L.simple_cubic(8, 8, 8, J=p["J"], k_u=0.0)
    m = {}
    for T in (0.5 * Tc, 1.5 * Tc):
        s = oracle_mod.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, 0.0, lat.easy_axis,
                                    alpha=p["lambda"], dt=p["dt_s"], seed=7)
        S, _ = oracle_mod.heun_run(s, L.uniform_state(lat.n), 4000, T)
        S, rec = oracle_mod.heun_run(s, S, 6000, T, step0=4000, record=True)
        m[T] = (np.linalg.norm(rec[:, :3], axis=1) / rec[:, 3]).mean()
    # ordered at Tc/2 (the fitted law (1 - T/Tc)^beta gives 0.79), disordered at 1.5 Tc
    # (only the finite-size |m| ~ N^-1/2 of 512 spins remains)
    assert 0.65 < m[0.5 * Tc] < 0.9, m
    assert m[1.5 * Tc] < 0.2, m

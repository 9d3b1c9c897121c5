"""Pins of the oracle's Hinzke-Nowak Monte Carlo step (Section "Monte Carlo Methods").

The equilibrium checks come from closed forms the Metropolis criterion (Eq. AMCP) must
reproduce for any mixture of symmetric trial moves:
  * the paper's Boltzmann distribution of a single spin with uniaxial anisotropy
    (Eq. boltz), which the paper offers as the test of the LLG "or Monte Carlo" integrator;
  * the Langevin function for free spins in a field, <S.h> = coth(x) - 1/x;
  * a classical Heisenberg dimer, <S1.S2> = coth(K) - 1/K with K = J/(kB T): a bond
    counted twice would give coth(2K) - 1/(2K);
  * the paper's fitted m(T) = (1 - T/Tc)^beta, Tc = 631.82 K, beta = 0.334297, for the
    simple-cubic ferromagnet of Fig. MCLLG (J = 6.0e-21 J/link, periodic, 21,952 atoms).
The move mixture (spin flip / Gaussian / random, Eqs. MCgaussian, MCrandom) is pinned by
one step of free spins, where every move is accepted and each kind is recognisable, and
the cone width Eq. MCgaussianSigma by its T^(1/5) scaling.
"""
import numpy as np
import pytest
from scipy import integrate

from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

KB = 1.3807e-23
MU_B = 9.2740e-24


def _free_spins(n, mu=1.5 * MU_B, k_u=0.0):
    return L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                         np.full(n, mu), np.full(n, k_u), np.tile([0.0, 0.0, 1.0], (n, 1)))


def _dimers(npairs, J, mu=1.5 * MU_B):
    n = 2 * npairs
    row_ptr = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32) ^ 1  # 0<->1, 2<->3, ...
    return L.SpinLattice(row_ptr, col.astype(np.int32), np.full(n, J), np.full(n, mu), np.zeros(n),
                         np.tile([0.0, 0.0, 1.0], (n, 1)))


def _langevin(x):
    return 1.0 / np.tanh(x) - 1.0 / x


def test_colouring_is_proper_and_a_checkerboard_on_even_simple_cubic(oracle_mod):
    lat = L.simple_cubic(6, 4, 8)
    colour, nc = oracle_mod.colour_greedy(oracle_system(lat))
    assert nc == 2
    idx = np.arange(lat.n)
    z = idx % 8
    x = (idx // 8) % 6
    y = idx // 48
    assert np.array_equal(colour, (x + y + z) % 2)
    for latc in (L.fcc(3, 3, 3), L.core_shell_sphere(diameter=2.4e-9, r_core=1.0e-9), L.simple_cubic(5, 5, 5)):
        colour, nc = oracle_mod.colour_greedy(oracle_system(latc))
        rows = np.repeat(np.arange(latc.n), np.diff(latc.row_ptr))
        assert not np.any(colour[rows] == colour[latc.col])
        assert colour.min() == 0 and colour.max() == nc - 1


def test_cone_width_scales_as_T_to_the_fifth(oracle_mod):
    T1 = MU_B / KB  # kB T / muB = 1
    assert oracle_mod.mc_sigma_g(T1) == pytest.approx(2.0 / 25.0, rel=1e-14)
    for T in (10.0, 300.0, 1000.0):
        assert oracle_mod.mc_sigma_g(32.0 * T) / oracle_mod.mc_sigma_g(T) == pytest.approx(2.0, rel=1e-13)


def test_move_mixture_of_one_step_on_free_spins(oracle_mod):
    """J = k_u = H = 0: every trial has dE = 0 and is accepted.  Spin flips give -S
    exactly, random moves are uniform on the sphere, Gaussian moves stay within a cone of
    width sigma_g around S (Eq. MCgaussian): each kind is about a third of the moves."""
    n = 30000
    T = 10.0
    lat = _free_spins(n)
    sysm = oracle_system(lat, seed=21)
    S0 = L.random_state(n, 5)
    S1, _, acc = oracle_mod.mc_run(sysm, S0, 1, T)
    assert acc[0] == n
    dot = np.einsum("ij,ij->i", S0, S1)
    flip = np.all(S1 == -S0, axis=1)
    sg = oracle_mod.mc_sigma_g(T)
    assert sg == pytest.approx(0.08 * (KB * T / MU_B) ** 0.2)
    near = (~flip) & (dot > np.cos(5 * sg))
    far = ~(flip | near)
    # a random move lands inside the 5-sigma cone with probability (1 - cos(5 sg))/2
    p_cap = (1 - np.cos(5 * sg)) / 2
    third = n / 3
    assert abs(flip.sum() - third) < 5 * np.sqrt(n * 2 / 9)
    assert abs(near.sum() - third * (1 + p_cap)) < 5 * np.sqrt(n * 2 / 9) + 10
    # random moves outside the cap: S1.S0 uniform on [-1, c], c = cos(5 sigma_g)
    d_far = dot[far]
    c = np.cos(5 * sg)
    assert abs(d_far.mean() - (c - 1) / 2) < 5 * np.sqrt((1 + c) ** 2 / 12 / d_far.size)
    assert abs((d_far ** 2).mean() - (c ** 3 + 1) / (3 * (c + 1))) < 0.02
    # Gaussian moves: 1 - cos(angle) ~ sigma_g^2 (for a 3D Gaussian displacement of width
    # sigma_g added to a unit vector, E[1 - cos] ~ sigma_g^2 to leading order)
    ang = 1 - dot[near]
    assert 0.5 * sg ** 2 < ang.mean() < 1.5 * sg ** 2


@pytest.mark.parametrize("K", [1.0, 5.0])
def test_boltzmann_distribution_of_a_single_spin_with_anisotropy(oracle_mod, K):
    """Eq. boltz: P(theta) ~ sin(theta) exp(-K sin^2(theta)), K = k_u/(kB T); folded about
    pi/2.  Many non-interacting spins, each a single-spin system."""
    n, T = 4000, 50.0
    ku = K * KB * T
    lat = _free_spins(n, k_u=ku)
    sysm = oracle_system(lat, seed=3)
    S, _, _ = oracle_mod.mc_run(sysm, L.uniform_state(n), 100, T)
    samples = []
    step = 100
    for _ in range(20):
        S, _, _ = oracle_mod.mc_run(sysm, S, 10, T, step0=step)
        step += 10
        samples.append(np.abs(S[:, 2]))
    c = np.concatenate(samples)  # |cos theta|
    # analytic distribution of x = |cos theta| on [0, 1]: p(x) ~ exp(-K (1 - x^2))
    Z = integrate.quad(lambda x: np.exp(-K * (1 - x * x)), 0, 1)[0]
    mean_c2 = integrate.quad(lambda x: x * x * np.exp(-K * (1 - x * x)), 0, 1)[0] / Z
    assert abs((c ** 2).mean() - mean_c2) < 0.01
    edges = np.linspace(0, 1, 11)
    hist = np.histogram(c, bins=edges)[0] / c.size
    exact = np.array([integrate.quad(lambda x: np.exp(-K * (1 - x * x)), a, b)[0] / Z
                      for a, b in zip(edges[:-1], edges[1:])])
    assert np.abs(hist - exact).max() < 0.012


def test_free_spins_in_a_field_follow_the_langevin_function(oracle_mod):
    n, T = 4000, 100.0
    mu = 1.5 * MU_B
    x = 2.0
    H = (x * KB * T / mu) * np.array([0.6, 0.0, 0.8])
    lat = _free_spins(n, mu=mu)
    sysm = oracle_system(lat, H=tuple(H), seed=8)
    S, _, _ = oracle_mod.mc_run(sysm, L.random_state(n, 2), 60, T)
    proj = []
    step = 60
    for _ in range(20):
        S, _, _ = oracle_mod.mc_run(sysm, S, 5, T, step0=step)
        step += 5
        proj.append(S @ (H / np.linalg.norm(H)))
    assert abs(np.concatenate(proj).mean() - _langevin(x)) < 0.01


def test_heisenberg_dimer_counts_each_bond_once(oracle_mod):
    npairs, T, K = 3000, 100.0, 1.5
    lat = _dimers(npairs, J=K * KB * T)
    sysm = oracle_system(lat, seed=13)
    S, _, _ = oracle_mod.mc_run(sysm, L.random_state(2 * npairs, 4), 60, T)
    vals = []
    step = 60
    for _ in range(20):
        S, _, _ = oracle_mod.mc_run(sysm, S, 5, T, step0=step)
        step += 5
        vals.append(np.einsum("ij,ij->i", S[0::2], S[1::2]))
    got = np.concatenate(vals).mean()
    assert abs(got - _langevin(K)) < 0.015
    assert abs(got - _langevin(2 * K)) > 0.1


def test_zero_temperature_steps_never_raise_the_energy(oracle_mod):
    lat = L.simple_cubic(6, 6, 6, J=6.0e-21, k_u=1.0e-23)
    sysm = oracle_system(lat, H=(0.0, 0.3, 0.5), seed=2)
    _, rec, acc = oracle_mod.mc_run(sysm, L.random_state(lat.n, 7), 6, 0.0, record=True)
    E = rec[:, 7]
    assert np.all(np.diff(E) <= 1e-30)
    assert acc[0] > 0


@pytest.mark.parametrize("T,tol", [(300.0, 0.03), (450.0, 0.04)])
def test_magnetisation_matches_the_papers_fitted_curve(oracle_mod, T, tol):
    """Fig. MCLLG: sc, J = 6.0e-21 J/link, periodic, 21,952 = 28^3 atoms; the paper fits
    its Monte Carlo m(T) with (1 - T/Tc)^beta, Tc = 631.82 K, beta = 0.334297."""
    lat = L.simple_cubic(28, 28, 28, J=6.0e-21, k_u=0.0)
    sysm = oracle_system(lat, seed=31)
    oracle_mod.set_threads(oracle_mod.max_threads())
    try:
        S, _, _ = oracle_mod.mc_run(sysm, L.uniform_state(lat.n), 400, T)
        _, rec, _ = oracle_mod.mc_run(sysm, S, 400, T, step0=400, record=True)
    finally:
        oracle_mod.set_threads(1)
    m = np.linalg.norm(rec[:, :3], axis=1) / rec[:, 3]
    assert abs(m.mean() - (1 - T / 631.82) ** 0.334297) < tol

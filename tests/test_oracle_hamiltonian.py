"""Pins of the oracle's Hamiltonian, effective field and reductions.

* Energy: compared with a dense brute-force sum over unordered pairs i<j (each bond once,
  Eq. HJij under the single-count reading), uniaxial anisotropy, Zeeman and Neel terms.
* Field: compared with -(1/mu_s) dE/dS_i (Eq. Heff) taken by central finite differences of
  that brute-force energy, which catches a dropped term, a wrong sign or factor 2.
* Neel tensor: on a fully coordinated fcc site sum_j e_ij e_ij^T = 4 I, so the surface
  term is isotropic (constant energy, field parallel to S, no torque).
* Mean-field exchange relation (Eq. JijTc) reproduces Table II.
"""
import json
import os

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _random_system(oracle_mod, n=9, seed=3, neel=True):
    rng = np.random.default_rng(seed)
    # random symmetric sparse exchange with mixed signs
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < 0.5:
                A[i, j] = A[j, i] = rng.normal(0, 5e-21)
    row_ptr = [0]
    col, J = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        rng.shuffle(nz)
        col += list(nz)
        J += list(A[i, nz])
        row_ptr.append(len(col))
    mu = rng.uniform(1.0, 3.0, n) * L.MU_B
    ku = rng.normal(0, 2e-23, n)
    ax = rng.normal(size=(n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    K = None
    if neel:
        K = np.zeros((n, 6))
        for i in range(0, n, 2):
            M = rng.normal(0, 1e-23, (3, 3))
            M = M + M.T
            K[i] = [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]
    H = rng.normal(0, 3.0, 3)
    sysm = oracle_mod.OracleSystem(np.array(row_ptr), np.array(col), np.array(J), mu, ku, ax, K,
                                   H_app=tuple(H))
    return sysm, A, mu, ku, ax, K, H


def _brute_energy(S, A, mu, ku, ax, K, H):
    n = S.shape[0]
    eex = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            eex -= A[i, j] * S[i] @ S[j]
    ean = -np.sum(ku * np.einsum("ij,ij->i", S, ax) ** 2)
    if K is not None:
        for i in range(n):
            M = np.array([[K[i, 0], K[i, 3], K[i, 4]], [K[i, 3], K[i, 1], K[i, 5]], [K[i, 4], K[i, 5], K[i, 2]]])
            ean -= S[i] @ M @ S[i]
    eap = -np.sum(mu * (S @ H))
    return eex, ean, eap


def test_energy_matches_bruteforce_pair_sum(oracle_mod):
    sysm, A, mu, ku, ax, K, H = _random_system(oracle_mod)
    S = L.random_state(sysm.n, 11)
    out = oracle_mod.moment_energy(sysm, S)
    eex, ean, eap = _brute_energy(S, A, mu, ku, ax, K, H)
    np.testing.assert_allclose(out[4:7], [eex, ean, eap], rtol=1e-12, atol=1e-35)
    np.testing.assert_allclose(out[7], eex + ean + eap, rtol=1e-12)
    np.testing.assert_allclose(out[:3], (mu[:, None] * S).sum(0), rtol=1e-12)
    np.testing.assert_allclose(out[3], mu.sum(), rtol=1e-14)


def test_field_is_negative_energy_gradient_over_mu(oracle_mod):
    sysm, A, mu, ku, ax, K, H = _random_system(oracle_mod)
    S = L.random_state(sysm.n, 12)
    Hf = oracle_mod.fields(sysm, S)
    h = 1e-6
    for i in range(sysm.n):
        for c in range(3):
            Sp = S.copy(); Sp[i, c] += h
            Sm = S.copy(); Sm[i, c] -= h
            dE = (sum(_brute_energy(Sp, A, mu, ku, ax, K, H)) - sum(_brute_energy(Sm, A, mu, ku, ax, K, H))) / (2 * h)
            ref = -dE / mu[i]
            assert abs(Hf[i, c] - ref) <= 1e-7 * max(1.0, np.abs(Hf[i]).max()), (i, c, Hf[i, c], ref)


def test_cube_reductions_exact(oracle_mod):
    """2x2x2 free cube: each site has 3 neighbours, 12 bonds; hand-checkable states."""
    lat = L.simple_cubic(2, 2, 2, periodic=(False, False, False), J=6e-21, k_u=1e-23)
    assert lat.nnz == 24 and np.all(np.diff(lat.row_ptr) == 3)
    sysm = oracle_mod.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis,
                                   H_app=(0.0, 0.0, 2.0))
    # all up: 12 bonds -> E_exc = -12 J; E_ani = -8 ku; E_app = -8 mu H
    out = oracle_mod.moment_energy(sysm, L.uniform_state(8))
    mu = 1.5 * L.MU_B
    np.testing.assert_allclose(out, [0, 0, 8 * mu, 8 * mu, -12 * 6e-21, -8e-23, -16 * mu,
                                     -12 * 6e-21 - 8e-23 - 16 * mu], rtol=1e-14, atol=1e-40)
    # Neel state (checkerboard): every bond antiparallel -> E_exc = +12 J, M = 0
    S = L.uniform_state(8).copy()
    idx = np.arange(8)
    z, x, y = idx % 2, (idx // 2) % 2, idx // 4
    S[(x + y + z) % 2 == 1] *= -1
    out = oracle_mod.moment_energy(sysm, S)
    np.testing.assert_allclose(out[[0, 1, 2, 4, 5, 6]], [0, 0, 0, 12 * 6e-21, -8e-23, 0], atol=1e-40, rtol=1e-14)


def test_neel_full_coordination_is_isotropic(oracle_mod):
    lat = L.fcc(3, 3, 3, with_pos=True)
    ks = 5e-23
    # periodic minimum-image bond vectors: every site has 12 neighbours
    n = lat.n
    rows = np.repeat(np.arange(n), np.diff(lat.row_ptr))
    box = 3 * lat.meta["a"]
    d = lat.pos[lat.col] - lat.pos[rows]
    d -= box * np.round(d / box)
    K = np.zeros((n, 6))
    e = d / np.linalg.norm(d, axis=1, keepdims=True)
    comps = np.stack([e[:, 0] ** 2, e[:, 1] ** 2, e[:, 2] ** 2, e[:, 0] * e[:, 1], e[:, 0] * e[:, 2],
                      e[:, 1] * e[:, 2]], 1)
    np.add.at(K, rows, comps)
    K *= 0.5 * ks
    np.testing.assert_allclose(K[:, :3], 2 * ks, rtol=1e-12)
    np.testing.assert_allclose(K[:, 3:], 0, atol=1e-12 * ks)
    # and the generator's own routine gives the same tensor for a site with 12 neighbours
    sphere = L.core_shell_sphere(diameter=3e-9, k_s=ks, z_full=13)  # mark every site
    full = np.diff(sphere.row_ptr) == 12
    assert full.any()
    np.testing.assert_allclose(sphere.K_neel[full][:, :3], 2 * ks, rtol=1e-12)
    np.testing.assert_allclose(sphere.K_neel[full][:, 3:], 0, atol=1e-12 * ks)
    # isotropic tensor: energy -2 ks per site for any state, field parallel to S
    sysm = oracle_mod.OracleSystem(lat.row_ptr, lat.col, np.zeros_like(lat.J), lat.mu_s, np.zeros(n),
                                   lat.easy_axis, K)
    S = L.random_state(n, 5)
    out = oracle_mod.moment_energy(sysm, S)
    np.testing.assert_allclose(out[5], -2 * ks * n, rtol=1e-12)
    Hf = oracle_mod.fields(sysm, S)
    np.testing.assert_allclose(np.cross(S, Hf), 0, atol=1e-9)


def test_exchange_from_curie_temperature_matches_table_II():
    """Eq. JijTc, J = 3 kB Tc/(epsilon z), reproduces Table II's exchange constants."""
    kB = GOLD["table_I_constants"]["k_B"]
    for el, v in GOLD["table_II_elements"].items():
        if el == "cite":
            continue
        J = 3 * kB * v["Tc"] / (v["epsilon"] * v["z"])
        assert abs(J - v["J"]) / v["J"] < 2e-3, (el, J, v["J"])


def test_lattice_csr_invariants():
    for lat, z in ((L.simple_cubic(5, 4, 3), 6), (L.fcc(3, 2, 2), 12)):
        assert np.all(np.diff(lat.row_ptr) == z)
        rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
        assert np.all(lat.col != rows)
        fwd = set(zip(rows.tolist(), lat.col.tolist()))
        assert all((j, i) in fwd for i, j in fwd)
    f = L.film(16, 8, 4)
    counts = np.bincount(np.diff(f.row_ptr))
    assert counts[5] == 2 * 16 * 8 and counts[6] == 2 * 16 * 8 and f.nnz == 16 * 8 * (2 * 5 + 2 * 6)

"""The seeded synthetic workloads that stand in for the paper's systems (no GPU): the sizes and
structure of the thin film, the fcc crystal, the core-shell sphere and the grain ensemble, and the
neighbour-list invariants the library relies on (J_ij = J_ji, no self or repeated bonds)."""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L


def _rows(lat):
    return np.repeat(np.arange(lat.n, dtype=np.int64), np.diff(lat.row_ptr))


def _check_csr(lat):
    rows = _rows(lat)
    col = lat.col.astype(np.int64)
    assert (col != rows).all(), "self bond"
    fwd = rows * lat.n + col
    assert np.unique(fwd).size == fwd.size, "repeated bond"
    rev = col * lat.n + rows
    of, orv = np.argsort(fwd), np.argsort(rev)
    np.testing.assert_array_equal(fwd[of], rev[orv])  # every bond i -> j has its j -> i
    np.testing.assert_array_equal(lat.J[of], lat.J[orv])  # with the same J


def test_film_structure_and_full_size_count():
    nx, ny, nz = 64, 48, 16
    lat = L.film(nx, ny, nz)
    assert lat.n == nx * ny * nz
    z = np.diff(lat.row_ptr)
    layer = np.arange(lat.n) % nz  # z fastest
    assert (z[(layer == 0) | (layer == nz - 1)] == 5).all()  # free surfaces: one out-of-plane bond
    assert (z[(layer > 0) & (layer < nz - 1)] == 6).all()
    assert lat.nnz == nx * ny * (6 * nz - 2)
    assert lat.nnz / lat.n == 5.875
    _check_csr(lat)
    # periodic in-plane: site (x = 0, y = 0, z = 3) bonds to x = nx - 1 and y = ny - 1
    i = 3
    nb = set(lat.col[lat.row_ptr[i]:lat.row_ptr[i + 1]].tolist())
    assert 3 + nz * (nx - 1) in nb and 3 + nz * nx * (ny - 1) in nb
    # the benchmark's 1024 x 1024 x 16 film, by the same count
    assert 1024 * 1024 * (6 * 16 - 2) == 98_566_144
    assert np.allclose(lat.J, 6.0e-21) and np.allclose(lat.mu_s, 1.5 * L.MU_B) and np.allclose(lat.k_u, 1e-24)


def test_fcc_crystal():
    big = L.fcc(64, 64, 64)
    assert big.n == 1_048_576 and big.nnz == 12_582_912
    assert (np.diff(big.row_ptr) == 12).all()
    assert np.allclose(big.J, 11.2e-21) and np.allclose(big.mu_s, 1.72 * L.MU_B)
    _check_csr(L.fcc(6, 5, 4))


def test_core_shell_sphere():
    lat = L.core_shell_sphere()
    assert lat.n == 382_761
    z = np.diff(lat.row_ptr)
    assert z.min() == 6 and z.max() == 12
    _check_csr(lat)
    # bond values by the ends' region: core-core, shell-shell, core-shell
    core = np.einsum("ij,ij->i", lat.pos, lat.pos) < (8e-9) ** 2
    rows = _rows(lat)
    a, b = core[rows], core[lat.col]
    np.testing.assert_allclose(lat.J[a & b], 11.2e-21)
    np.testing.assert_allclose(lat.J[~a & ~b], -5.0e-21)
    np.testing.assert_allclose(lat.J[a != b], 2.0e-21)
    assert lat.meta["n_core"] == int(core.sum())
    # Neel tensors on the 25,554 under-coordinated sites only, trace (k_s / 2) z_i there
    surf = z < 12
    assert surf.sum() == 25_554 == lat.meta["n_surface"]
    assert not lat.K_neel[~surf].any()
    np.testing.assert_allclose(lat.K_neel[surf, :3].sum(1), 0.5 * 5.0e-23 * z[surf], rtol=1e-12)
    assert np.allclose(lat.mu_s, 1.72 * L.MU_B) and not lat.k_u.any()


@pytest.fixture(scope="module")
def grains():
    return L.grain_ensemble(count=256, seed=12345)


def test_grain_ensemble(grains):
    gs, temps = grains
    sizes = np.array([g.n for g in gs])
    assert len(gs) == 256 and sizes.sum() == 5_184_550
    assert sizes.min() >= 2000 and sizes.max() <= 40000
    assert (sizes % 10 == 0).all()  # columns extruded over 10 layers
    assert temps.min() >= 0.0 and temps.max() <= 800.0
    ku = np.array([g.k_u[0] for g in gs])
    assert all(np.all(g.k_u == g.k_u[0]) for g in gs)  # one k_u per grain
    assert abs(ku.mean() / 1e-23 - 1) < 0.06  # log-normal, arithmetic mean 1e-23 (standard error ~2 %)
    assert abs(np.log(ku).std() - 0.3) < 0.05
    ez = np.array([g.easy_axis[0, 2] for g in gs])
    assert (ez >= np.cos(np.deg2rad(5.0)) - 1e-12).all()  # easy axes within 5 degrees of +z
    for g in gs[:8]:
        assert np.diff(g.row_ptr).max() <= 6  # simple cubic with free surfaces
        _check_csr(g)

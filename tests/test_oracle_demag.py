"""Pins of the oracle's macrocell demagnetising field (Section "Demagnetising fields",
Eqs. macrocellpos, mc_volume, demag).

  * one macrocell holding every atom: the field is the self term -mu0 M/3 exactly;
  * two point dipoles: the field on the dipole axis is -2 times the broadside field, falls
    as 1/r^3, and the interaction is reciprocal (m1.H_12 = m2.H_21);
  * a uniformly magnetised sphere: -mu0 M/3 inside (demagnetising factor 1/3);
  * the paper's 20 nm x 20 nm x 1 nm platelet magnetised out of plane with macrocells of two
    unit cells: about -mu0 M at the centre (the paper: -2.236 T against -mu0 M = -2.18 T);
  * the paper's prolate ellipsoid (fcc, a = 3.54 A, 1.5 muB, 10 nm x 20 nm, macrocells of two
    unit cells): the shape-anisotropy shift Delta N mu0 Ms, Delta N = N_x - N_z from the mean
    field over the atoms, against the paper's simulated 0.33 T (Osborn's continuum value for an
    axis ratio of 2 gives 0.37 T; the paper's macrocell result, like this one, lies below it);
  * the update interval (reading D4): one run of 10 steps equals two runs of 5 when the field
    is updated every 5 steps, and differs from updating every step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L

MU0 = 4e-7 * np.pi
MU_B = 9.2740e-24


def _points(pos, mu, cell, vatom):
    n = len(pos)
    return O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                          np.broadcast_to(mu, (n,)), np.zeros(n), (0, 0, 1), pos=pos, demag_cell=cell,
                          demag_vatom=vatom)


def _sc_points(nx, ny, nz, a):
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    return g.astype(np.float64) * a


def test_single_macrocell_gives_the_self_term_exactly():
    a, mu = 3e-10, 2.0 * MU_B
    pos = _sc_points(4, 4, 4, a)
    s = _points(pos, mu, cell=10 * a, vatom=a ** 3)
    S = L.random_state(len(pos), 3)
    Hd, Hmc = O.demag_fields(s, S)
    assert Hmc.shape == (1, 3)
    M = mu * S.sum(axis=0) / (len(pos) * a ** 3)
    np.testing.assert_allclose(Hmc[0], -MU0 / 3 * M, rtol=1e-13)
    assert np.all(Hd == Hmc[0])


def test_point_dipoles_axis_broadside_ratio_scaling_and_reciprocity():
    a, mu, vat = 3e-10, 1.5 * MU_B, (3e-10) ** 3
    for d in (5e-9, 10e-9):
        pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
        s = _points(pos, mu, cell=a, vatom=vat)
        self_z = -MU0 / 3 * mu / vat
        Hax, _ = O.demag_fields(s, np.array([[0, 0, 1.0], [0, 0, 1.0]]))  # moments along the axis
        Hbr, _ = O.demag_fields(s, np.array([[1.0, 0, 0], [1.0, 0, 0]]))  # broadside
        axial = Hax[0, 2] - self_z
        broad = Hbr[0, 0] - self_z
        # (the self term is ~1e4 times the dipole field here: the subtraction costs four digits)
        assert axial / broad == pytest.approx(-2.0, rel=1e-9)
        if d == 5e-9:
            axial5 = axial
        else:
            assert axial5 / axial == pytest.approx(8.0, rel=1e-9)
    # reciprocity with different moments and directions
    pos = np.array([[0.0, 0.0, 0.0], [3e-9, -2e-9, 4e-9]])
    s = O.OracleSystem(np.zeros(3, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                       np.array([1.5, 2.5]) * MU_B, np.zeros(2), (0, 0, 1), pos=pos, demag_cell=a, demag_vatom=vat)
    S = L.random_state(2, 8)
    H, _ = O.demag_fields(s, S)
    m = S * (np.array([1.5, 2.5]) * MU_B)[:, None]
    self_ = -MU0 / 3 * m / vat
    assert m[0] @ (H[0] - self_[0]) == pytest.approx(m[1] @ (H[1] - self_[1]), rel=1e-9, abs=0)


def test_uniform_sphere_has_demagnetising_factor_one_third():
    a, mu = 2.5e-10, 2.0 * MU_B
    R = 6e-9
    g = _sc_points(49, 49, 49, a) - 24 * a
    pos = g[np.linalg.norm(g, axis=1) <= R]
    s = _points(pos, mu, cell=2 * a, vatom=a ** 3)
    Hd, _ = O.demag_fields(s, L.uniform_state(len(pos)))
    M = mu / a ** 3
    centre = np.linalg.norm(pos, axis=1) < 2 * a
    assert Hd[centre, 2].mean() / (-MU0 * M) == pytest.approx(1 / 3, rel=0.03)
    assert np.abs(Hd[centre, :2]).max() < 1e-3 * MU0 * M


def test_paper_platelet_centre_field_is_about_minus_mu0_M():
    a, mu = 2.5e-10, 2.22 * MU_B
    pos = _sc_points(80, 80, 4, a)  # 20 nm x 20 nm x 1 nm
    s = _points(pos, mu, cell=2 * a, vatom=a ** 3)
    Hd, _ = O.demag_fields(s, L.uniform_state(len(pos)))
    M = mu / a ** 3
    c = np.linalg.norm(pos[:, :2] - 39.5 * a, axis=1) < 2 * a
    ratio = Hd[c, 2].mean() / (-MU0 * M)
    assert 0.97 < ratio < 1.08  # the paper's own calculation: 2.236 / 2.18 = 1.026
    edge = pos[:, 0] < a / 2
    assert Hd[edge, 2].mean() > 0.8 * Hd[c, 2].mean()  # weaker (less negative) at the edges


def test_paper_prolate_ellipsoid_shape_anisotropy():
    a, mu = 3.54e-10, 1.5 * MU_B
    nc = 32
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(-nc, nc)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + base[None]) * a).reshape(-1, 3)
    # diameter 10 nm across (x, y), height 20 nm along z
    inside = (pos[:, 0] / 5e-9) ** 2 + (pos[:, 1] / 5e-9) ** 2 + (pos[:, 2] / 10e-9) ** 2 <= 1.0
    pos = pos[inside]
    s = _points(pos, mu, cell=2 * a, vatom=a ** 3 / 4)
    M = 4 * mu / a ** 3
    Hz, _ = O.demag_fields(s, L.uniform_state(len(pos)))
    Sx = np.zeros((len(pos), 3))
    Sx[:, 0] = 1.0
    Hx, _ = O.demag_fields(s, Sx)
    Nz = -Hz[:, 2].mean() / (MU0 * M)
    Nx = -Hx[:, 0].mean() / (MU0 * M)
    m = 2.0  # axis ratio
    Nz_ref = (m / np.sqrt(m * m - 1) * np.log(m + np.sqrt(m * m - 1)) - 1) / (m * m - 1)
    Nx_ref = (1 - Nz_ref) / 2
    assert Nx_ref - Nz_ref == pytest.approx(0.2397, abs=5e-4)
    assert (Nx_ref - Nz_ref) * MU0 * M == pytest.approx(0.37, abs=0.01)  # the paper's expected shift
    # the macrocell scheme's shift sits where the paper's simulation put it (0.33 T), below
    # the continuum value, as the paper found
    shift = (Nx - Nz) * MU0 * M
    assert shift == pytest.approx(0.33, rel=0.08)
    assert 0.75 * 0.37 < shift < 0.37


def test_update_interval_holds_the_field_between_updates():
    lat = L.simple_cubic(8, 8, 2, periodic=(False, False, False), J=6e-21, k_u=0.0, with_pos=True)
    mk = lambda every: O.OracleSystem(  # noqa: E731
        lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.5, dt=1e-15, seed=5,
        pos=lat.pos, demag_cell=6e-10, demag_vatom=(3e-10) ** 3, demag_every=every)
    S0 = L.random_state(lat.n, 1)
    one, _ = O.heun_run(mk(5), S0, 10, 50.0)
    half, _ = O.heun_run(mk(5), S0, 5, 50.0)
    two, _ = O.heun_run(mk(5), half, 5, 50.0, step0=5)
    assert np.array_equal(one, two)
    every1, _ = O.heun_run(mk(1), S0, 10, 50.0)
    assert np.abs(every1 - one).max() > 1e-9
    off = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.5, dt=1e-15,
                         seed=5)
    none, _ = O.heun_run(off, S0, 10, 50.0)
    assert np.abs(none - one).max() > 1e-6


@pytest.mark.parametrize("scheme", ["midpoint", "semi_implicit"])
def test_alternative_integrators_hold_the_field_and_agree_with_heun(scheme):
    """The midpoint rule and the semi-implicit scheme take the held field as the Heun step
    does (reading D4): one run of 10 steps equals two of 5 with updates every 5, and with the
    field updated every step their difference from the Heun trajectory falls as dt^2 (a field
    left out or taken at another state would leave an O(1) difference)."""
    lat = L.simple_cubic(8, 8, 2, periodic=(False, False, False), J=6e-21, k_u=0.0, with_pos=True)
    mk = lambda every, dt, J=1.0: O.OracleSystem(  # noqa: E731
        lat.row_ptr, lat.col, J * lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.5, dt=dt, seed=5, pos=lat.pos,
        demag_cell=6e-10, demag_vatom=(3e-10) ** 3, demag_every=every)
    if scheme == "midpoint":
        run = lambda s, S, n, st=0: O.midpoint_run(s, S, n, 0.0, iters=30, step0=st)  # noqa: E731
    else:
        run = lambda s, S, n, st=0: O.sib_run(s, S, n, 0.0, step0=st)  # noqa: E731
    S0 = L.random_state(lat.n, 1)
    one, _ = run(mk(5, 1e-15), S0, 10)
    half, _ = run(mk(5, 1e-15), S0, 5)
    two, _ = run(mk(5, 1e-15), half, 5, 5)
    assert np.array_equal(one, two)
    # with exchange (20 fs), and with the demagnetising field as the only field (40 ps)
    for J, dts, t_end in ((1.0, (4e-16, 2e-16, 1e-16), 2e-14), (0.0, (2e-13, 1e-13, 5e-14), 4e-11)):
        d = []
        for dt in dts:
            nst = int(round(t_end / dt))
            a, _ = run(mk(1, dt, J), S0, nst)
            b, _ = O.heun_run(mk(1, dt, J), S0, nst, 0.0)
            d.append(np.abs(a - b).max())
        assert 3.5 < d[0] / d[1] < 4.5 and 3.5 < d[1] / d[2] < 4.5

"""The long-range fcc builder (exchange to every site within r_cut, the shape of the paper's
long-ranged exchange with over 1,000 neighbours per atom), checked against brute force over
site positions.

  * neighbour counts per shell against the fcc shell sequence (12, 6, 24, 12, 24, 8, 48, ...)
    and the total within 4a (1,060), from a direct enumeration of lattice points;
  * every bond's length is its J's shell distance, J decreases with distance, the bonds of a
    bulk site sum to J_total, and every bond has its reverse with the same J;
  * free surfaces: a site's row holds exactly the sites of the finite crystal within r_cut,
    found by brute force over all pairs.
"""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L


def test_shell_counts_against_enumeration():
    st = L.fcc_stencil(4.0)
    assert st.shape[0] == 1060
    n2 = (st * st).sum(axis=1)
    counts = [int((n2 == k).sum()) for k in sorted(set(n2.tolist()))]
    assert counts[:8] == [12, 6, 24, 12, 24, 8, 48, 6]
    # brute force: points of the cubic-cell lattice plus basis, at distance <= 4a
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(-5, 6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pts = (cells[:, None, :] + base[None]).reshape(-1, 3)
    d = np.linalg.norm(pts, axis=1)
    assert int(((d > 0) & (d <= 4.0 + 1e-9)).sum()) == 1060


def test_bonds_lengths_values_and_symmetry():
    lat = L.fcc_long_range(9, 9, 9, r_cut=4.0, with_pos=True)
    a = lat.meta["a"]
    n = lat.n
    assert n == 4 * 9 ** 3 and np.all(np.diff(lat.row_ptr) == 1060)
    rows = np.repeat(np.arange(n), np.diff(lat.row_ptr))
    box = np.array(lat.meta["cells"]) * a
    d = lat.pos[lat.col] - lat.pos[rows]
    d -= box * np.round(d / box)  # minimum image
    r = np.linalg.norm(d, axis=1) / a
    assert r.max() <= 4.0 + 1e-12 and r.min() == pytest.approx(1 / np.sqrt(2), rel=1e-12)
    expect = lat.J[0] * np.exp(-(r - 1 / np.sqrt(2)) / 0.5)
    np.testing.assert_allclose(lat.J, expect, rtol=1e-12)
    assert lat.J[lat.row_ptr[0]:lat.row_ptr[1]].sum() == pytest.approx(12 * 11.2e-21, rel=1e-13)
    # distinct targets within each row, no self bonds, and every bond's reverse with the same J
    for i in (0, 1, 777, n - 1):
        c = lat.col[lat.row_ptr[i]:lat.row_ptr[i + 1]]
        assert np.unique(c).size == c.size and i not in c
    key = rows * n + lat.col
    rkey = lat.col.astype(np.int64) * n + rows
    order = np.argsort(key)
    pos = np.searchsorted(key[order], rkey)
    assert np.array_equal(key[order][pos], rkey)
    assert np.array_equal(lat.J[order][pos], lat.J)


def test_free_surfaces_against_all_pairs():
    lat = L.fcc_long_range(4, 3, 5, r_cut=1.6, periodic=(False, False, False), with_pos=True)
    a = lat.meta["a"]
    D = np.linalg.norm(lat.pos[:, None, :] - lat.pos[None, :, :], axis=2) / a
    for i in range(lat.n):
        want = np.nonzero((D[i] > 0) & (D[i] <= 1.6 + 1e-9))[0]
        got = np.sort(lat.col[lat.row_ptr[i]:lat.row_ptr[i + 1]])
        assert np.array_equal(got, want)
    lens = np.diff(lat.row_ptr)
    assert lens.min() < lens.max()  # ragged rows at the surfaces


def test_periodic_box_must_exceed_twice_the_cutoff():
    with pytest.raises(ValueError):
        L.fcc_long_range(8, 9, 9, r_cut=4.0)

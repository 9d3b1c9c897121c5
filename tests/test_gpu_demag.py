"""Parity of the CUDA macrocell demagnetising field (through the C ABI) with the oracle,
and of the Heun-LLG step that uses it.

FP64: the per-atom field matches the oracle's within 1e-12 of its largest component (the
cell centres and moments are summed in the same order; the pair sums differ only in the
rounding of 1/r), and trajectories with the field updated every k steps match within
1e-12.  FP32-mixed: the moments come from FP32 spins and the field is applied in FP32,
1e-6 relative on the field and 1e-4 on trajectories.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi
MU_B = 9.2740e-24


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _oracle(lat, cell, vatom, every=1, **kw):
    return O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel,
                          pos=lat.pos, demag_cell=cell, demag_vatom=vatom, demag_every=every, **kw)


def _lat(nx=12, ny=10, nz=4, a=3e-10):
    lat = L.simple_cubic(nx, ny, nz, periodic=(False, False, False), J=6e-21, k_u=1e-23, a=a, with_pos=True)
    lat.mu_s = lat.mu_s * (1.0 + 0.3 * (np.arange(lat.n) % 3 == 0))  # two moments: weighted centres matter
    return lat


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_field_matches_oracle(SS, precision, tol):
    a = 3e-10
    lat = _lat(a=a)
    S = L.random_state(lat.n, 4)
    S[:, 2] += 0.8
    S /= np.linalg.norm(S, axis=1, keepdims=True)
    with SS(lat, T=0.0, S0=S, precision=precision) as s:
        s.set_demag(2.5 * a, a ** 3, every=10)
        H = s.demag_field()
    Href, _ = O.demag_fields(_oracle(lat, 2.5 * a, a ** 3), S)
    assert np.abs(H - Href).max() <= tol * np.abs(Href).max()


def test_batch_fields_do_not_cross_systems(SS):
    a = 3e-10
    lats = [_lat(8, 8, 3, a), _lat(6, 5, 4, a)]
    Ss = [L.random_state(l.n, 10 + k) for k, l in enumerate(lats)]
    with SS(lats, T=0.0, S0=Ss, precision="fp64") as b:
        b.set_demag(2 * a, a ** 3)
        Hb = b.demag_field()
    off = 0
    for lat, S in zip(lats, Ss):
        Href, _ = O.demag_fields(_oracle(lat, 2 * a, a ** 3), S)
        assert np.abs(Hb[off:off + lat.n] - Href).max() <= 1e-12 * np.abs(Href).max()
        off += lat.n


@pytest.mark.parametrize("every", [1, 5])
def test_fp64_trajectory_with_held_field_matches_oracle(SS, every):
    a = 3e-10
    lat = _lat(10, 10, 3, a)
    S0 = L.random_state(lat.n, 7)
    kw = dict(alpha=0.3, dt=2e-16, seed=5)
    with SS(lat, T=100.0, S0=S0, precision="fp64", **kw) as s:
        s.set_demag(2 * a, a ** 3, every=every)
        s.step(60)
        S_gpu = s.spins()
        rec = s.record(0, 60)
    S_ref, rec_ref = O.heun_run(_oracle(lat, 2 * a, a ** 3, every=every, **kw), S0, 60, 100.0, record=True)
    assert np.abs(S_gpu - S_ref).max() <= 1e-12
    assert np.abs(rec[:, 0, 7] - rec_ref[:, 7]).max() <= 1e-12 * np.abs(rec_ref[:, 7]).max()


def test_fp32_trajectory_with_field(SS):
    a = 3e-10
    lat = _lat(10, 10, 3, a)
    S0 = L.random_state(lat.n, 7)
    kw = dict(alpha=0.3, dt=2e-16, seed=5)
    with SS(lat, T=100.0, S0=S0, precision="fp32", **kw) as s:
        s.set_demag(2 * a, a ** 3, every=5)
        s.step(50)
        S_gpu = s.spins()
    S_ref, _ = O.heun_run(_oracle(lat, 2 * a, a ** 3, every=5, **kw), S0, 50, 100.0)
    assert np.abs(S_gpu - S_ref).max() <= 1e-4


def test_graph_and_persistent_modes_equal_plain_launches(SS):
    a = 3e-10
    lat = _lat(16, 16, 4, a)
    S0 = L.random_state(lat.n, 2)
    out = {}
    for mode in ("kernels", "graph", "persistent"):
        with SS(lat, T=300.0, S0=S0, precision="fp32", seed=3) as s:
            s.set_exec(mode)
            s.set_demag(2 * a, a ** 3, every=20)
            s.step(130)
            out[mode] = s.spins()
    assert np.array_equal(out["kernels"], out["graph"])
    assert np.array_equal(out["kernels"], out["persistent"])


def test_field_is_refreshed_after_set_spins_and_switched_off(SS):
    a = 3e-10
    lat = _lat(8, 8, 2, a)
    with SS(lat, T=0.0, precision="fp64") as s:
        s.set_demag(2 * a, a ** 3, every=1000)
        H_up = s.demag_field()
        S = L.random_state(lat.n, 1)
        s.set_spins(S)
        H_new = s.demag_field()
        Href, _ = O.demag_fields(_oracle(lat, 2 * a, a ** 3), S)
        assert np.abs(H_new - Href).max() <= 1e-12 * np.abs(Href).max()
        assert np.abs(H_new - H_up).max() > 1e-3
        s.set_demag(0.0, 0.0)
        with pytest.raises(Exception):
            s.demag_field()


def test_needs_positions(SS):
    lat = L.simple_cubic(4, 4, 4)
    with SS(lat, T=0.0) as s:
        with pytest.raises(Exception, match="positions"):
            s.set_demag(6e-10, 2.7e-29)


def test_paper_platelet_and_ellipsoid_through_the_library(SS):
    """The paper's 20 x 20 x 1 nm platelet (about -mu0 M at the centre) and prolate
    ellipsoid (shape shift against the paper's simulated 0.33 T), as in the oracle pins."""
    a, mu = 2.5e-10, 2.22 * MU_B
    g = np.stack(np.meshgrid(np.arange(80), np.arange(80), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    pos = g.astype(np.float64) * a
    n = len(pos)
    plate = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, mu),
                          np.zeros(n), np.tile([0.0, 0.0, 1.0], (n, 1)), pos=pos)
    with SS(plate, T=0.0, precision="fp64") as s:
        s.set_demag(2 * a, a ** 3)
        H = s.demag_field()
    c = np.linalg.norm(pos[:, :2] - 39.5 * a, axis=1) < 2 * a
    assert 0.97 < H[c, 2].mean() / (-MU0 * mu / a ** 3) < 1.08
    a, mu = 3.54e-10, 1.5 * MU_B
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(-32, 32)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + base[None]) * a).reshape(-1, 3)
    pos = pos[(pos[:, 0] / 5e-9) ** 2 + (pos[:, 1] / 5e-9) ** 2 + (pos[:, 2] / 10e-9) ** 2 <= 1.0]
    n = len(pos)
    ell = L.SpinLattice(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), np.full(n, mu),
                        np.zeros(n), np.tile([0.0, 0.0, 1.0], (n, 1)), pos=pos)
    Sx = np.tile([1.0, 0.0, 0.0], (n, 1))
    with SS(ell, T=0.0, precision="fp64") as s:
        s.set_demag(2 * a, a ** 3 / 4)
        Hz = s.demag_field()
        s.set_spins(Sx)
        Hx = s.demag_field()
    shift = Hz[:, 2].mean() - Hx[:, 0].mean()  # (N_x - N_z) mu0 M, since H_k = -N_k mu0 M
    assert shift == pytest.approx(0.33, rel=0.08)


@pytest.mark.parametrize("scheme", ["midpoint", "semi_implicit"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_alternative_integrators_with_the_field_match_oracle(SS, scheme, precision, tol):
    """The midpoint rule and the semi-implicit scheme with the field updated every 5 steps,
    then Heun steps from a multiple of the interval (the oracle recomputes the field at the
    first step of each run, the library at multiples of the interval), against the oracle."""
    a = 3e-10
    lat = _lat(10, 10, 3, a)
    S0 = L.random_state(lat.n, 9)
    kw = dict(alpha=0.3, dt=2e-16, seed=6)
    with SS(lat, T=100.0, S0=S0, precision=precision, **kw) as s:
        s.set_demag(2 * a, a ** 3, every=5)
        if scheme == "midpoint":
            s.midpoint_step(20, iterations=3)
        else:
            s.semi_implicit_step(20)
        s.step(5)
        S_gpu = s.spins()
        rec = s.record(0, 25)
    ref = _oracle(lat, 2 * a, a ** 3, every=5, **kw)
    if scheme == "midpoint":
        S_ref, r1 = O.midpoint_run(ref, S0, 20, 100.0, iters=3, record=True)
    else:
        S_ref, r1 = O.sib_run(ref, S0, 20, 100.0, record=True)
    S_ref, r2 = O.heun_run(ref, S_ref, 5, 100.0, step0=20, record=True)
    assert np.abs(S_gpu - S_ref).max() <= tol
    if precision == "fp64":
        rr = np.concatenate([r1, r2])
        assert np.abs(rec[:, 0, 7] - rr[:, 7]).max() <= 1e-12 * np.abs(rr[:, 7]).max()

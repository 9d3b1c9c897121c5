"""Parity of the CUDA path with the oracle on long exchange rows (1,060 neighbours per atom,
the shape of the paper's long-ranged exchange with over 1,000 neighbours), where the exchange
sum runs a warp per row (packed bond words, plain col + J, or tensors) ahead of each Heun pass.

FP64: trajectories and records within 1e-12 of the oracle after 100 steps at 300 K (the warp
sums its row in another order than the oracle's loop); the thread-per-row and warp-per-row
modes agree to the same bound.  FP32-mixed: 1e-4 over 100 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


@pytest.fixture(scope="module")
def lr9():
    return L.fcc_long_range(9, 9, 9, r_cut=4.0)


def _run(SS, lat, steps, precision, mode="auto", T=300.0, **kw):
    kw.setdefault("seed", 7)
    with SS(lat, alpha=0.1, dt=1e-16, T=T, precision=precision, **kw) as s:
        if mode != "auto":
            s.set_exchange_rows(mode)
        info = s.info()
        s.step(steps)
        return s.spins(), s.record(0, steps), info


def _check_records(rec, rec_ref):
    g = rec[:, 0, :]
    assert np.abs(g[:, :4] - rec_ref[:, :4]).max() <= 1e-12 * np.abs(rec_ref[:, 3]).max()
    assert np.abs(g[:, 4:] - rec_ref[:, 4:]).max() <= 1e-12 * np.abs(rec_ref[:, 4]).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_packed_warp_rows_match_oracle(SS, lr9, precision, tol):
    S0 = L.random_state(lr9.n, 3)
    S, rec, info = _run(SS, lr9, 100, precision, S0=S0, H=(0.0, 0.3, 0.5), sys_id=4)
    assert info["exchange_rows"] == 3  # a warp per row, packed bonds
    S_ref, rec_ref = O.heun_run(oracle_system(lr9, H=(0.0, 0.3, 0.5), seed=7, sys_id=4), S0, 100, 300.0,
                                record=True)
    assert np.abs(S - S_ref).max() <= tol
    if precision == "fp64":
        _check_records(rec, rec_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sliced_rows_equal_thread_rows_bitwise(SS, lr9, precision):
    """The sliced pass sums each row in its CSR order from H_app, as a thread per row does:
    the trajectories and records are identical."""
    S0 = L.random_state(lr9.n, 5)
    Sw, rw, iw = _run(SS, lr9, 60, precision, S0=S0)
    St, rt, it = _run(SS, lr9, 60, precision, mode="thread", S0=S0)
    assert iw["exchange_rows"] == 3 and it["exchange_rows"] == 1
    assert np.array_equal(Sw, St) and np.array_equal(rw, rt)


def test_warp_rows_agree_with_thread_rows(SS):
    # short rows forced onto a warp each (uniform J, no packed words)
    sc = L.simple_cubic(12, 12, 12, J=6e-21, k_u=1e-23)
    S0 = L.random_state(sc.n, 6)
    Sw, _, iw = _run(SS, sc, 80, "fp64", mode="warp", S0=S0)
    St, _, it = _run(SS, sc, 80, "fp64", S0=S0)
    assert iw["exchange_rows"] == 2 and it["exchange_rows"] == 1
    assert np.abs(Sw - St).max() <= 1e-12


def test_free_surfaces_ragged_rows_match_oracle(SS):
    lat = L.fcc_long_range(7, 7, 8, r_cut=3.0, periodic=(False, True, False))
    lens = np.diff(lat.row_ptr)
    assert lens.min() < lens.max() and lat.nnz >= 64 * lat.n
    S0 = L.random_state(lat.n, 8)
    S, rec, info = _run(SS, lat, 80, "fp64", S0=S0, T=500.0)
    assert info["exchange_rows"] == 3
    S_ref, rec_ref = O.heun_run(oracle_system(lat, seed=7), S0, 80, 500.0, record=True)
    assert np.abs(S - S_ref).max() <= 1e-12
    _check_records(rec, rec_ref)


def test_unpacked_and_tensor_rows_match_oracle(SS):
    lat = L.fcc_long_range(9, 9, 9, r_cut=3.0)
    # more than 256 distinct J values: bond-symmetric random factors, read as col + J
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    lo, hi = np.minimum(rows, lat.col), np.maximum(rows, lat.col)
    f = 0.5 + ((lo * 2654435761 + hi * 40503) % 1000) / 1000.0
    lat.J = lat.J * f
    S0 = L.random_state(lat.n, 9)
    S, rec, info = _run(SS, lat, 60, "fp64", S0=S0)
    assert info["exchange_rows"] == 2
    S_ref, rec_ref = O.heun_run(oracle_system(lat, seed=7), S0, 60, 300.0, record=True)
    assert np.abs(S - S_ref).max() <= 1e-12
    _check_records(rec, rec_ref)
    # exchange tensors with an interface-type DM part on every long-range bond
    lt = L.with_dm(L.fcc_long_range(9, 9, 9, r_cut=3.0, with_pos=True), 1e-21)
    lt.k_c = np.full(lt.n, 1e-23)
    S0 = L.random_state(lt.n, 10)
    S, _, info = _run(SS, lt, 50, "fp64", S0=S0)
    assert info["exchange_rows"] == 2
    ref = O.OracleSystem(lt.row_ptr, lt.col, lt.J, lt.mu_s, lt.k_u, lt.easy_axis, lt.K_neel, alpha=0.1, dt=1e-16,
                         seed=7, J_tensor=lt.J_tensor, k_c=lt.k_c)
    S_ref, _ = O.heun_run(ref, S0, 50, 300.0)
    assert np.abs(S - S_ref).max() <= 1e-12


def test_batch_with_short_rows_and_temperatures(SS, lr9):
    sc = L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23)
    lats = [lr9, sc]
    S0s = [L.random_state(l.n, 20 + k) for k, l in enumerate(lats)]
    temps = [700.0, 100.0]
    with SS(lats, alpha=0.1, dt=1e-16, T=temps, seed=[1, 2], sys_id=[0, 1], S0=S0s, precision="fp64") as b:
        assert b.info()["exchange_rows"] == 3
        b.step(40)
        S_b = b.spins()
        E = [b.energy(k) for k in range(2)]
    off = 0
    for k, lat in enumerate(lats):
        ref = oracle_system(lat, seed=k + 1, sys_id=k)
        S_ref, _ = O.heun_run(ref, S0s[k], 40, temps[k])
        assert np.abs(S_b[off:off + lat.n] - S_ref).max() <= 1e-12
        e_ref = O.moment_energy(ref, S_ref)
        assert E[k][0] == pytest.approx(e_ref[7], rel=1e-12, abs=0)
        off += lat.n


def test_exec_modes_and_graphs(SS, lr9):
    S0 = L.random_state(lr9.n, 11)
    out = {}
    for mode in ("kernels", "graph"):
        with SS(lr9, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=3, precision="fp32") as s:
            s.set_exec(mode)
            s.step(70)
            out[mode] = s.spins()
            with pytest.raises(Exception, match="graph or plain"):
                s.set_exec("persistent")
            s.set_exchange_rows("thread")
            s.set_exec("persistent")
            s.set_exchange_rows("warp")
            assert s.info()["exec"] == 0
    assert np.array_equal(out["kernels"], out["graph"])


def test_edge_cases_empty_rows_and_single_spins(SS, lr9):
    """A batch mixing long rows with bond-free spins and a one-spin system: the slices holding
    empty rows are padded, the free spins precess in the applied field alone; FP64 parity."""
    free = L.SpinLattice(np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                         np.full(5, 2 * 9.274e-24), np.full(5, 1e-23), np.tile([0.0, 0.0, 1.0], (5, 1)))
    one = L.SpinLattice(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0),
                        np.full(1, 2 * 9.274e-24), np.zeros(1), np.tile([0.0, 0.0, 1.0], (1, 1)))
    lats = [free, lr9, one]
    S0s = [L.random_state(l.n, 30 + k) for k, l in enumerate(lats)]
    temps = [50.0, 300.0, 0.0]
    H = [(0.0, 0.0, 1.0), (0.2, 0.0, 0.0), (1.0, 0.0, 0.0)]
    with SS(lats, alpha=0.1, dt=1e-16, T=temps, H=H, seed=[4, 5, 6], sys_id=[0, 1, 2], S0=S0s,
            precision="fp64") as b:
        assert b.info()["exchange_rows"] == 3
        b.step(30)
        S_b = b.spins()
        rec = b.record(0, 30)
    off = 0
    for k, lat in enumerate(lats):
        ref = oracle_system(lat, H=H[k], seed=k + 4, sys_id=k)
        S_ref, rec_ref = O.heun_run(ref, S0s[k], 30, temps[k], record=True)
        assert np.abs(S_b[off:off + lat.n] - S_ref).max() <= 1e-12
        assert np.abs(rec[:, k, 7] - rec_ref[:, 7]).max() <= 1e-12 * max(np.abs(rec_ref[:, 7]).max(), 1e-30)
        off += lat.n


@pytest.mark.parametrize("scheme", ["midpoint", "semi_implicit"])
def test_alternative_integrators_on_long_rows(SS, scheme):
    """The midpoint rule and the semi-implicit scheme read their exchange sums from the row
    passes: FP64 parity with the oracle, and bitwise the thread-per-row result with packed
    slices (same summation order)."""
    lat = L.fcc_long_range(9, 9, 9, r_cut=3.0)
    S0 = L.random_state(lat.n, 13)

    def run(mode, precision="fp64"):
        with SS(lat, alpha=0.1, dt=1e-16, T=300.0, S0=S0, seed=3, precision=precision) as s:
            if mode != "auto":
                s.set_exchange_rows(mode)
            if scheme == "midpoint":
                s.midpoint_step(30, iterations=3)
            else:
                s.semi_implicit_step(30)
            return s.spins(), s.record(0, 30), s.info()["exchange_rows"]

    Sw, rw, mw = run("auto")
    St, rt, mt = run("thread")
    assert mw == 3 and mt == 1
    assert np.array_equal(Sw, St) and np.array_equal(rw, rt)
    ref = oracle_system(lat, seed=3)
    if scheme == "midpoint":
        S_ref, _ = O.midpoint_run(ref, S0, 30, 300.0, iters=3)
    else:
        S_ref, _ = O.sib_run(ref, S0, 30, 300.0)
    assert np.abs(Sw - S_ref).max() <= 1e-12
    S32, _, _ = run("auto", "fp32")
    assert np.abs(S32 - S_ref).max() <= 1e-4


@pytest.mark.parametrize("kind", ["long_range", "forced_warp_sc"])
def test_monte_carlo_on_long_rows(SS, kind):
    """Monte Carlo with a warp summing the rows of 32 trials: FP64 per-step accepted counts
    equal to the oracle's and spins within 1e-12 (the row sums differ only in order)."""
    if kind == "long_range":
        lat = L.fcc_long_range(9, 9, 9, r_cut=3.0)
        mode, steps, T = "auto", 8, 900.0
    else:
        lat = L.simple_cubic(8, 8, 8, J=6e-21, k_u=1e-23)
        mode, steps, T = "warp", 20, 400.0
    S0 = L.random_state(lat.n, 21)
    with SS(lat, alpha=0.1, dt=1e-16, T=T, S0=S0, seed=5, sys_id=1, precision="fp64") as s:
        if mode != "auto":
            s.set_exchange_rows(mode)
        assert s.info()["exchange_rows"] >= 2
        accs, prev = [], 0
        for _ in range(steps):
            s.mc_step(1)
            acc, _ = s.mc_stats(0)
            accs.append(acc - prev)
            prev = acc
        S = s.spins()
        rec = s.record(0, steps)
    S_ref, rec_ref, acc_ref = O.mc_run(oracle_system(lat, seed=5, sys_id=1), S0, steps, T, record=True)
    assert np.array_equal(np.array(accs), acc_ref)
    assert np.abs(S - S_ref).max() <= 1e-12
    assert np.abs(rec[:, 0, 7] - rec_ref[:, 7]).max() <= 1e-12 * np.abs(rec_ref[:, 7]).max()


def test_monte_carlo_long_rows_fp32_warp_and_thread_agree(SS):
    """FP32-mixed Monte Carlo on long rows: the warp-summed passes (their trial randoms drawn for
    all spins by a pass of their own) against the thread-per-row passes (each trial drawing its
    own): the same moves and thresholds, row sums in another order."""
    lat = L.fcc_long_range(9, 9, 9, r_cut=3.0)
    S0 = L.random_state(lat.n, 4)
    out = {}
    for mode in ("warp", "thread"):
        with SS(lat, alpha=0.1, dt=1e-16, T=700.0, S0=S0, seed=9, precision="fp32") as s:
            s.set_exchange_rows(mode)
            s.mc_step(6)
            out[mode] = (s.spins(), s.mc_stats(0)[0])
    acc_w, acc_t = out["warp"][1], out["thread"][1]
    assert abs(acc_w - acc_t) <= 0.002 * lat.n * 6, (acc_w, acc_t)
    same = np.all(out["warp"][0] == out["thread"][0], axis=1).mean()
    assert same > 0.99, same

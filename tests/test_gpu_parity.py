"""Parity of the CUDA Heun-LLG path (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated by the benchmark spec): FP64 path max|dS| <= 1e-12 after 1000 steps of the
10x10x10 simple-cubic configuration; FP32-mixed path max|dS| <= 1e-4 over 100 steps.
Moments and energies: relative 1e-12 (FP64) / 1e-5 (FP32-mixed; the per-spin terms are
FP32 products summed in FP64).
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import oracle_system

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _compare_records(rec_gpu, rec_ref, rtol):
    # rec_gpu: (steps, 1, 8); rec_ref: (steps, 8)
    g = rec_gpu[:, 0, :]
    scale_m = np.abs(rec_ref[:, 3]).max()
    scale_e = np.abs(rec_ref[:, 4:7]).max()
    assert np.abs(g[:, :4] - rec_ref[:, :4]).max() <= rtol * scale_m
    assert np.abs(g[:, 4:] - rec_ref[:, 4:]).max() <= rtol * scale_e


def test_sc10_fp64_1000_steps(SS):
    """Configuration: sc 10^3 periodic, J = 6e-21, mu_s = 1.5 muB, k_u = 1e-24 || z,
    H = 0, alpha = 0.1, dt = 1e-16 s, T = 300 K, all spins +z, seed 1, FP64."""
    lat = L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24)
    with SS(lat, alpha=0.1, dt=1e-16, T=300.0, seed=1, precision="fp64") as s:
        s.step(1000)
        S_gpu = s.spins()
        rec = s.record(0, 1000)
        m_now = s.magnetisation()
        e_now = s.energy()
    ref = oracle_system(lat, alpha=0.1, dt=1e-16, seed=1)
    S_ref, rec_ref = O.heun_run(ref, L.uniform_state(lat.n), 1000, 300.0, record=True)
    assert np.abs(S_gpu - S_ref).max() <= TOL64
    _compare_records(rec, rec_ref, TOL64)
    me = O.moment_energy(ref, S_ref)
    np.testing.assert_allclose(m_now[:3], me[:3] / me[3], atol=TOL64)
    np.testing.assert_allclose(e_now, [me[7], me[4], me[5], me[6]], rtol=1e-11, atol=1e-11 * abs(me[4]))


def test_sc10_fp32_100_steps(SS):
    lat = L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24)
    with SS(lat, alpha=0.1, dt=1e-16, T=300.0, seed=1, precision="fp32") as s:
        s.step(100)
        S_gpu = s.spins()
        rec = s.record(0, 100)
    S_ref, rec_ref = O.heun_run(oracle_system(lat), L.uniform_state(lat.n), 100, 300.0, record=True)
    assert np.abs(S_gpu - S_ref).max() <= TOL32
    _compare_records(rec, rec_ref, 1e-5)


@pytest.mark.parametrize("precision,tol,steps", [("fp64", TOL64, 300), ("fp32", TOL32, 100)])
def test_all_terms_ragged_tiles(SS, precision, tol, steps):
    """Every Hamiltonian term at once: random easy axes, applied field, Neel tensors on
    the surface of a small core-shell sphere (irregular rows), with a system size that
    leaves a ragged last tile."""
    lat = L.core_shell_sphere(diameter=3.2e-9, r_core=1.2e-9, k_s=5e-23)
    rng = np.random.default_rng(4)
    ax = rng.normal(size=(lat.n, 3))
    lat.easy_axis = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    lat.k_u = rng.uniform(0, 5e-23, lat.n)
    assert lat.n % 128 != 0 and lat.n > 3 * 256
    S0 = L.random_state(lat.n, 9)
    H = (0.7, -0.2, 1.0)
    with SS(lat, alpha=0.2, dt=5e-17, T=150.0, H=H, seed=77, sys_id=5, S0=S0, precision=precision) as s:
        s.set_launch(128, 128)
        s.step(steps)
        S_gpu = s.spins()
        rec = s.record(0, steps)
    ref = oracle_system(lat, alpha=0.2, dt=5e-17, H=H, seed=77, sys_id=5)
    S_ref, rec_ref = O.heun_run(ref, S0, steps, 150.0, record=True)
    assert np.abs(S_gpu - S_ref).max() <= tol
    _compare_records(rec, rec_ref, 1e-12 if precision == "fp64" else 1e-5)


def test_exec_modes_bitwise_identical(SS):
    lat = L.simple_cubic(9, 7, 5)
    out = {}
    for mode in ("kernels", "graph", "persistent", "system_blocks", "cluster"):
        with SS(lat, alpha=0.1, dt=1e-16, T=400.0, seed=3, precision="fp64") as s:
            s.set_launch(128, 256)
            s.set_exec(mode)
            s.step(130)
            out[mode] = (s.spins(), s.record(0, 130))
    for mode in ("graph", "persistent", "cluster"):
        np.testing.assert_array_equal(out[mode][0], out["kernels"][0])
        np.testing.assert_array_equal(out[mode][1], out["kernels"][1])
    # whole systems per block: same spins; the record sums in another order
    np.testing.assert_array_equal(out["system_blocks"][0], out["kernels"][0])
    np.testing.assert_allclose(out["system_blocks"][1], out["kernels"][1], rtol=1e-13,
                               atol=1e-13 * np.abs(out["kernels"][1]).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_many_small_systems_one_block_each(SS, precision):
    """A temperature sweep of 300 small lattices (sizes 27..729, ragged against the block)
    advanced with one thread block per system equals the per-step launches, and its
    systems match the oracle."""
    lats = [L.simple_cubic(3 + k % 7, 3 + (k // 7) % 5, 3 + k % 3) for k in range(300)]
    kw = dict(alpha=0.1, dt=1e-16, T=[float(3 * k) for k in range(300)], seed=[7 + k for k in range(300)],
              sys_id=list(range(300)))
    res = {}
    for mode in ("kernels", "system_blocks"):
        with SS(lats, precision=precision, **kw) as s:
            s.set_launch(128, 128)
            s.set_exec(mode)
            s.step(37)
            res[mode] = (s.spins(), s.record(0, 37), s.step_index)
    np.testing.assert_array_equal(res["system_blocks"][0], res["kernels"][0])
    assert res["system_blocks"][2] == 37
    np.testing.assert_allclose(res["system_blocks"][1], res["kernels"][1], rtol=1e-12,
                               atol=1e-12 * np.abs(res["kernels"][1]).max())
    if precision == "fp64":
        off = 0
        for k in (0, 151, 299):
            off = sum(l.n for l in lats[:k])
            S_ref, _ = O.heun_run(oracle_system(lats[k], seed=7 + k, sys_id=k), L.uniform_state(lats[k].n), 37,
                                  3.0 * k)
            assert np.abs(res["system_blocks"][0][off:off + lats[k].n] - S_ref).max() <= TOL64


def test_launch_shapes_agree(SS):
    """Tile and block shapes change only the summation order of the reductions."""
    lat = L.fcc(4, 3, 3)
    base = None
    for block, tile in ((128, 128), (256, 512), (512, 2048)):
        with SS(lat, alpha=0.05, dt=1e-16, T=500.0, seed=8, precision="fp64") as s:
            s.set_launch(block, tile)
            s.step(50)
            cur = (s.spins(), s.record(0, 50))
        if base is None:
            base = cur
        else:
            np.testing.assert_array_equal(cur[0], base[0])
            np.testing.assert_allclose(cur[1], base[1], rtol=1e-13, atol=1e-13 * np.abs(base[1]).max())


def test_batch_equals_unbatched(SS):
    lats = [L.simple_cubic(6, 5, 4), L.fcc(2, 2, 3), L.single_spin(k_u=2e-23), L.simple_cubic(3, 3, 3)]
    kw = dict(alpha=[0.1, 0.05, 0.3, 1.0], dt=[1e-16, 1e-16, 2e-16, 5e-17], T=[300.0, 0.0, 50.0, 900.0],
              H=[(0, 0, 1.0), (0.5, 0, 0), (0, 0, 0), (0, 1.0, 0)], seed=[1, 2, 3, 1], sys_id=[0, 1, 2, 3])
    with SS(lats, precision="fp64", **kw) as b:
        b.step(64)
        Sb = b.spins()
        rb = b.record(0, 64)
    for k, lat in enumerate(lats):
        single = {key: v[k] for key, v in kw.items()}
        with SS(lat, precision="fp64", **single) as s:
            s.step(64)
            Ss = s.spins()
            rs = s.record(0, 64)
        off = sum(l.n for l in lats[:k])
        np.testing.assert_array_equal(Sb[off:off + lat.n], Ss)
        np.testing.assert_array_equal(rb[:, k, :], rs[:, 0, :])


def test_batch_matches_oracle_per_system(SS):
    lats = [L.simple_cubic(5, 5, 5), L.fcc(2, 2, 2)]
    with SS(lats, alpha=[0.1, 0.2], dt=1e-16, T=[250.0, 700.0], seed=[10, 11], sys_id=[4, 9], precision="fp64") as b:
        b.step(200)
        S = b.spins()
    off = 0
    for lat, a, T, sd, sid in zip(lats, (0.1, 0.2), (250.0, 700.0), (10, 11), (4, 9)):
        S_ref, _ = O.heun_run(oracle_system(lat, alpha=a, seed=sd, sys_id=sid), L.uniform_state(lat.n), 200, T)
        assert np.abs(S[off:off + lat.n] - S_ref).max() <= TOL64
        off += lat.n


def test_temperature_schedule(SS):
    lat = L.simple_cubic(6, 6, 6)
    nsteps = 150
    T = 300.0 + 900.0 * np.exp(-0.5 * ((np.arange(nsteps) - 60) / 15.0) ** 2)
    with SS(lat, alpha=0.02, dt=1e-16, seed=5, precision="fp64") as s:
        s.set_temperature_schedule(T, step0=0)
        s.step(nsteps)
        S = s.spins()
    S_ref, _ = O.heun_run(oracle_system(lat, alpha=0.02, seed=5), L.uniform_state(lat.n), nsteps, T)
    assert np.abs(S - S_ref).max() <= TOL64


def test_resume_is_bitwise(SS):
    lat = L.simple_cubic(5, 4, 6)
    with SS(lat, alpha=0.1, T=300.0, seed=2, precision="fp32") as s:
        s.step(1000)
        full = s.spins()
    with SS(lat, alpha=0.1, T=300.0, seed=2, precision="fp32") as s:
        s.step(500)
        mid = s.spins()
        step = s.step_index
    assert step == 500
    with SS(lat, alpha=0.1, T=300.0, seed=2, precision="fp32", S0=mid) as s:
        s.step_index = 500
        s.step(500)
        np.testing.assert_array_equal(s.spins(), full)


def test_single_spin_analytic_on_gpu(SS):
    """T = 0 single spin against Eq. analytic_LLG (the paper's 1e-6 bound at dt = 1 fs)."""
    lam, H, dt = 0.1, 10.0, 1e-15
    g = 1.76e11
    with SS(L.single_spin(), alpha=lam, dt=dt, T=0.0, H=(0, 0, H), S0=np.array([[1.0, 0, 0]]),
            precision="fp64") as s:
        err = 0.0
        for k in range(60):
            s.step(1000)
            t = (k + 1) * 1000 * dt
            a = lam * g * H / (1 + lam ** 2) * t
            w = g * H / (1 + lam ** 2) * t
            ref = np.array([np.cos(w) / np.cosh(a), np.sin(w) / np.cosh(a), np.tanh(a)])
            err = max(err, np.abs(s.spins()[0] - ref).max())
    assert 1e-8 < err < 1e-6


def test_init_random_matches_oracle_stream(SS):
    lat = L.fcc(3, 3, 3)
    for prec, tol in (("fp64", 1e-15), ("fp32", 1e-7)):
        with SS(lat, seed=2, sys_id=0, init_random=True, precision=prec) as s:
            S = s.spins()
        np.testing.assert_allclose(S, O.init_sphere(2, 0, lat.n), atol=tol)


def test_unit_length_and_nonfinite_flag(SS):
    from paper_1310_6143_gb300._binding import SpinSysError

    lat = L.simple_cubic(4, 4, 4)
    with SS(lat, T=2000.0, precision="fp32") as s:
        for _ in range(5):
            s.step(7)
            S = s.spins()
            np.testing.assert_allclose(np.linalg.norm(S, axis=1), 1.0, atol=3e-7)
    # an exchange so large that the FP32 field overflows: the kernel flags it
    huge = L.simple_cubic(4, 4, 4, J=1e30)
    with SS(huge, T=0.0, precision="fp32", S0=L.random_state(huge.n, 1)) as s:
        s.step(1)
        with pytest.raises(SpinSysError, match="NONFINITE"):
            s.sync()
        s.sync()  # the flag is cleared once reported


def test_barrier_timeout_reports_and_recovers(SS):
    from paper_1310_6143_gb300._binding import SpinSysError

    lat = L.simple_cubic(8, 8, 8)
    with SS(lat, T=300.0, precision="fp32") as s:
        s.set_exec("persistent")
        s.set_barrier_test(extra=1, timeout_ns=20_000_000)  # waits for a block that never comes
        s.step(3)
        with pytest.raises(SpinSysError, match="TIMEOUT"):
            s.sync()
        s.set_barrier_test(extra=0, timeout_ns=2_000_000_000)
        s.step_index = 0
        s.set_spins(L.uniform_state(lat.n))
        s.step(10)
        s.sync()
        assert s.step_index == 10


def test_validation_errors(SS):
    from paper_1310_6143_gb300._binding import SpinSysError

    lat = L.simple_cubic(3, 3, 3)
    bad = L.SpinLattice(lat.row_ptr, lat.col.copy(), lat.J, lat.mu_s, lat.k_u, lat.easy_axis)
    bad.col[5] = 999
    with pytest.raises(SpinSysError, match="INVALID_ARG"):
        SS(bad)
    with pytest.raises(SpinSysError, match="INVALID_ARG"):
        SS(lat, dt=-1.0)

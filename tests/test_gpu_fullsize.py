"""Full-size workloads in the benchmark's launch configuration, checked on samples.

For each workload the GPU takes one Heun step from a random state; sampled spins (bulk,
surfaces, the first and last sites, tile boundaries) are recomputed by the oracle from
their exact two-bond neighbourhood (the predictor values of the neighbours need their
own neighbours), with the Philox spin word mapped to the global index.  Properties that
hold at any size are checked on every spin: |S| = 1, and the step's record of the
initial state equals the oracle's FP64 moment and energy of that state.  The film is also
compared whole: all 16,777,216 spins after eight steps against the oracle run over the film.
"""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L
from tests._helpers import neighbourhood, oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


@pytest.fixture(scope="module")
def film():
    return L.film(1024, 1024, 16)


def _samples(n, tile, rng, extra=()):
    idx = {0, n - 1, tile - 1, tile, min(n - 1, 5 * tile + 3)}
    idx.update(int(v) for v in rng.integers(0, n, 24))
    idx.update(int(v) for v in extra)
    return np.array(sorted(i for i in idx if 0 <= i < n))


def _check_one_step(SS, lat, precision, tol, alpha, dt, T, H=(0.0, 0.0, 0.0), seed=5, extra=(), exec_mode="graph"):
    rng = np.random.default_rng(seed)
    S0 = L.random_state(lat.n, seed)
    with SS(lat, alpha=alpha, dt=dt, T=T, H=H, seed=seed, S0=S0, precision=precision) as s:
        s.set_exec(exec_mode)
        start = s.spins()  # the state as stored (rounded to FP32 in the mixed form)
        s.step(1)
        S1 = s.spins()
        rec = s.record(0, 1)[0, 0]
        tile = s.info()["tile"]
    np.testing.assert_allclose(np.linalg.norm(S1, axis=1), 1.0, atol=4e-7 if precision == "fp32" else 1e-15)
    ref = oracle_system(lat, alpha=alpha, dt=dt, H=H, seed=seed)
    me = O.moment_energy(ref, start)
    rtol = 1e-5 if precision == "fp32" else 1e-12
    assert abs(rec[3] - me[3]) <= 1e-14 * me[3]
    assert np.abs(rec[:3] - me[:3]).max() <= rtol * me[3]
    assert np.abs(rec[4:] - me[4:]).max() <= rtol * np.abs(me[4:7]).sum()
    samples = _samples(lat.n, tile, rng, extra)
    for c in samples:
        sites, sub = neighbourhood(lat, np.array([c]), 2)
        sref = oracle_system(sub, alpha=alpha, dt=dt, H=H, seed=seed, ids=sites.astype(np.uint32))
        out, _ = O.heun_run(sref, start[sites], 1, T, step0=0)
        k = int(np.searchsorted(sites, c))
        assert np.abs(out[k] - S1[c]).max() <= tol, (c, out[k], S1[c])


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-6), ("fp64", 1e-14)])
def test_film_1024x1024x16(SS, film, precision, tol):
    lat = film
    nz = 16
    surface = [3 * nz, 3 * nz + nz - 1, lat.n - 1 - nz * 1024]  # bottom / top layer sites
    _check_one_step(SS, lat, precision, tol, alpha=0.02, dt=1e-16, T=1200.0, extra=surface)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_film_whole_state_eight_steps_as_benchmarked(SS, film, precision, tol):
    """Every spin of the film after eight steps in the benchmark's execution mode (one launch
    of the captured eight-step graph that the library chooses for a system of this size,
    default launch shape, the corrector drawing part of the next step's thermal field) under a
    temperature pulse, against the oracle run over the whole film; the eight in-loop records of
    the pre-step states against the oracle's."""
    lat = film
    T = np.array([300.0, 450.0, 700.0, 1000.0, 1200.0, 1000.0, 700.0, 450.0])
    S0 = L.random_state(lat.n, 31)
    with SS(lat, alpha=0.02, dt=1e-16, T=0.0, seed=5, S0=S0, precision=precision) as s:
        s.set_temperature_schedule(T)
        start = s.spins()
        assert s.info()["exec"] == 0  # automatic: eight or more steps of a system this size run as a graph
        s.step(8)
        S = s.spins()
        rec = s.record(0, 8)[:, 0, :]
    ref = oracle_system(lat, alpha=0.02, dt=1e-16, seed=5)
    S_ref, rec_ref = O.heun_run(ref, start, 8, T, record=True)
    assert np.abs(S - S_ref).max() <= tol
    rtol = 1e-5 if precision == "fp32" else 1e-12
    ms = rec_ref[0, 3]
    assert np.abs(rec[:, 3] - rec_ref[:, 3]).max() <= 1e-14 * ms
    assert np.abs(rec[:, :3] - rec_ref[:, :3]).max() <= rtol * ms
    assert np.abs(rec[:, 4:] - rec_ref[:, 4:]).max() <= rtol * np.abs(rec_ref[:, 4:7]).sum(1).max()


def test_fcc_64_cubed(SS):
    lat = L.fcc(64, 64, 64)
    _check_one_step(SS, lat, "fp32", 2e-6, alpha=0.05, dt=1e-16, T=1500.0)


def test_core_shell_sphere_20nm(SS):
    lat = L.core_shell_sphere()
    surf = np.nonzero(np.diff(lat.row_ptr) < 12)[0][:8]
    _check_one_step(SS, lat, "fp32", 2e-6, alpha=0.1, dt=1e-16, T=10.0, H=(1.0, 0.0, 0.0), extra=surf)
    _check_one_step(SS, lat, "fp64", 1e-14, alpha=0.1, dt=1e-16, T=10.0, H=(1.0, 0.0, 0.0), extra=surf)


def test_grain_ensemble_256(SS):
    """256 grains in one batched persistent launch: each grain is checked against its
    own oracle system on sampled spins."""
    grains, temps = L.grain_ensemble(count=256, seed=12345)
    seeds = list(range(1000, 1256))
    S0 = [L.random_state(g.n, k) for k, g in enumerate(grains)]
    with SS(grains, alpha=0.1, dt=1e-16, T=list(temps), seed=seeds, S0=S0, precision="fp32") as s:
        s.set_exec("persistent")
        start = s.spins()
        s.step(1)
        S1 = s.spins()
        rec = s.record(0, 1)[0]
    np.testing.assert_allclose(np.linalg.norm(S1, axis=1), 1.0, atol=4e-7)
    rng = np.random.default_rng(1)
    off = np.cumsum([0] + [g.n for g in grains])
    for gidx in rng.choice(256, 12, replace=False):
        g = grains[gidx]
        o = off[gidx]
        ref = oracle_system(g, alpha=0.1, dt=1e-16, seed=seeds[gidx], sys_id=int(gidx))
        me = O.moment_energy(ref, start[o:o + g.n])
        assert np.abs(rec[gidx, :3] - me[:3]).max() <= 1e-5 * me[3]
        for c in rng.integers(0, g.n, 4):
            sites, sub = neighbourhood(g, np.array([c]), 2)
            sref = oracle_system(sub, alpha=0.1, dt=1e-16, seed=seeds[gidx], sys_id=int(gidx),
                                 ids=sites.astype(np.uint32))
            out, _ = O.heun_run(sref, start[o + sites], 1, temps[gidx])
            k = int(np.searchsorted(sites, c))
            assert np.abs(out[k] - S1[o + c]).max() <= 2e-6


def _whole_state(SS, lats, precision, steps, tol, oracles, T, **kw):
    """Autotune as the benchmark does (the state is restored), take `steps` steps, and compare
    every spin and every system's records with the oracle runs over the whole systems."""
    with SS(lats, precision=precision, T=T, **kw) as s:
        s.autotune(8)
        start = s.spins()
        s.step(steps)
        S = s.spins()
        rec = s.record(0, steps)
    temps = T if isinstance(T, list) else [T]
    rtol = 1e-5 if precision == "fp32" else 1e-12
    off = 0
    for k, (ref, n) in enumerate(oracles):
        S_ref, rec_ref = O.heun_run(ref, start[off:off + n], steps, temps[k], record=True)
        assert np.abs(S[off:off + n] - S_ref).max() <= tol, k
        ms = rec_ref[0, 3]
        assert np.abs(rec[:, k, 3] - rec_ref[:, 3]).max() <= 1e-14 * ms
        assert np.abs(rec[:, k, :3] - rec_ref[:, :3]).max() <= rtol * ms
        assert np.abs(rec[:, k, 4:] - rec_ref[:, 4:]).max() <= rtol * np.abs(rec_ref[:, 4:7]).sum(1).max()
        off += n


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_fcc64_whole_state_as_benchmarked(SS, precision, tol):
    """The fcc 64^3 crystal of the temperature sweep (random start from the library's reserved
    stream, 1,000 K), 64 steps (one captured graph) in the autotuned launch shape."""
    lat = L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24)
    ref = oracle_system(lat, alpha=0.05, dt=1e-16, seed=2)
    _whole_state(SS, lat, precision, 64, tol, [(ref, lat.n)], 1000.0, alpha=0.05, dt=1e-16, seed=2,
                 init_random=True)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_fcc64_dm_cubic_whole_state_as_benchmarked(SS, precision, tol):
    """fcc 64^3 with a DM term (|D| = 0.1 J, nine exchange values per bond) and cubic anisotropy
    at 300 K, 64 steps in the autotuned launch shape."""
    lat = L.with_dm(L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24, with_pos=True), D=1.12e-21)
    lat.k_c = np.full(lat.n, 5e-24)
    ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel, alpha=0.05,
                         dt=1e-16, seed=4, J_tensor=lat.J_tensor, k_c=lat.k_c)
    _whole_state(SS, lat, precision, 64, tol, [(ref, lat.n)], 300.0, alpha=0.05, dt=1e-16, seed=4,
                 init_random=True)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_core_shell_whole_state_as_benchmarked(SS, precision, tol):
    """The 20 nm core-shell sphere (Neel surface anisotropy, 1 T along x, 10 K), 64 steps in the
    autotuned launch shape."""
    lat = L.core_shell_sphere()
    S0 = L.random_state(lat.n, 33)
    ref = oracle_system(lat, alpha=0.1, dt=1e-16, H=(1.0, 0.0, 0.0), seed=3)
    _whole_state(SS, lat, precision, 64, tol, [(ref, lat.n)], 10.0, alpha=0.1, dt=1e-16, H=(1.0, 0.0, 0.0),
                 seed=3, S0=S0)


def test_grain_ensemble_whole_state_as_benchmarked(SS):
    """All 256 grains (5.2 M spins) of the batched form, FP32-mixed, 16 steps in the autotuned
    launch shape, every spin and every grain's records against one oracle run per grain."""
    grains, temps = L.grain_ensemble(count=256, seed=12345)
    seeds = [4000 + k for k in range(256)]
    S0 = [L.random_state(g.n, 50 + k) for k, g in enumerate(grains)]
    refs = [(oracle_system(g, alpha=0.1, dt=1e-16, seed=seeds[k], sys_id=k), g.n) for k, g in enumerate(grains)]
    _whole_state(SS, grains, "fp32", 16, 1e-4, refs, [float(t) for t in temps], alpha=0.1, dt=1e-16, seed=seeds,
                 sys_id=list(range(256)), S0=S0)

"""Parity of the CUDA path with the oracle for tensorial exchange (Eqs. HJijM, HJijSMS, with a
Dzyaloshinskii-Moriya part) and cubic anisotropy: FP64 Heun-LLG trajectories within 1e-12,
FP32-mixed within 1e-4, FP64 Monte Carlo with identical per-step acceptance; J times the
identity reproduces the scalar path bitwise; batches mixing tensor and scalar systems equal
each system alone; the symmetry check rejects tensors whose reverse bond is not the transpose."""
import numpy as np
import pytest

import oracle as O
from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu

MU_B = 9.2740e-24


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _skew(d):
    return np.array([[0.0, -d[2], d[1]], [d[2], 0.0, -d[0]], [-d[1], d[0], 0.0]])


def _tensor_lattice(nx, ny, nz, seed, J=6e-21):
    lat = L.simple_cubic(nx, ny, nz, J=J, k_u=5e-24)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    where = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(rows, lat.col))}
    Jt = np.zeros((lat.nnz, 3, 3))
    for k, (i, j) in enumerate(zip(rows, lat.col)):
        if i < j:
            B = rng.normal(size=(3, 3)) * 0.1 * J
            A = J * np.eye(3) + 0.5 * (B + B.T) + _skew(rng.normal(size=3) * 0.2 * J)
            Jt[k], Jt[where[(int(j), int(i))]] = A, A.T
    lat.J_tensor = Jt
    lat.k_c = rng.uniform(-3e-23, 3e-23, lat.n)
    lat.mu_s = lat.mu_s * rng.uniform(0.9, 1.1, lat.n)
    return lat


def _oracle(lat, **kw):
    return O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel,
                          J_tensor=lat.J_tensor, k_c=lat.k_c, **kw)


@pytest.mark.parametrize("precision,tol,steps", [("fp64", 1e-12, 200), ("fp32", 1e-4, 100)])
def test_llg_matches_oracle(SS, precision, tol, steps):
    lat = _tensor_lattice(6, 6, 6, 1)
    S0 = L.random_state(lat.n, 3)
    kw = dict(alpha=0.1, dt=1e-16, seed=7, sys_id=1, H=(0.2, 0.0, 0.5))
    with SS(lat, T=300.0, S0=S0, precision=precision, check_symmetry=True, **kw) as s:
        s.step(steps)
        S = s.spins()
        rec = s.record(0, steps)
    okw = dict(alpha=0.1, dt=1e-16, seed=7, sys_id=1, H_app=(0.2, 0.0, 0.5))
    S_ref, rec_ref = O.heun_run(_oracle(lat, **okw), S0, steps, 300.0, record=True)
    assert np.abs(S - S_ref).max() <= tol
    rtol = 1e-12 if precision == "fp64" else 1e-5
    assert np.abs(rec[:, 0, 4:] - rec_ref[:, 4:]).max() <= rtol * np.abs(rec_ref[:, 4:7]).max()


def test_monte_carlo_matches_oracle(SS):
    lat = _tensor_lattice(6, 6, 6, 2)
    S0 = L.random_state(lat.n, 4)
    with SS(lat, T=250.0, S0=S0, precision="fp64", seed=5) as s:
        accs, prev = [], 0
        for _ in range(20):
            s.mc_step(1)
            a, _ = s.mc_stats(0)
            accs.append(a - prev)
            prev = a
        S = s.spins()
    S_ref, _, acc_ref = O.mc_run(_oracle(lat, seed=5), S0, 20, 250.0)
    assert np.array_equal(np.array(accs), acc_ref)
    assert np.abs(S - S_ref).max() <= 1e-12


def test_identity_tensor_is_the_scalar_path_bitwise(SS):
    lat = L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23)
    tl = L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23)
    tl.J_tensor = lat.J[:, None, None] * np.eye(3)[None]
    out = []
    for la in (lat, tl):
        with SS(la, T=300.0, seed=2, precision="fp64") as s:
            s.step(50)
            s.mc_step(5)
            out.append(s.spins())
    assert np.array_equal(out[0], out[1])


def test_batch_of_tensor_and_scalar_systems_equals_each_alone(SS):
    lats = [_tensor_lattice(4, 4, 4, 3), L.simple_cubic(5, 4, 3, J=5e-21, k_u=1e-23)]
    with SS(lats, T=[200.0, 400.0], seed=[1, 2], sys_id=[0, 1], precision="fp64") as b:
        b.step(40)
        Sb = b.spins()
    off = 0
    for k, lat in enumerate(lats):
        with SS(lat, T=[200.0, 400.0][k], seed=k + 1, sys_id=k, precision="fp64") as s:
            s.step(40)
            assert np.abs(s.spins() - Sb[off:off + lat.n]).max() <= 1e-13
        off += lat.n


def test_symmetry_check_rejects_untransposed_tensors(SS):
    lat = _tensor_lattice(3, 3, 3, 4)
    lat.J_tensor = lat.J_tensor.copy()
    lat.J_tensor[0] = lat.J_tensor[0].T + 1e-22 * _skew([1.0, 0, 0])
    with pytest.raises(Exception, match="transposed"):
        SS(lat, T=0.0, check_symmetry=True)

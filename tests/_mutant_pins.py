"""Quick pins run against one (possibly mutated) oracle library in a child process.

Prints one line per pin, 'PASS name' or 'FAIL name'.  Used by test_oracle_mutants.py.
"""
import math
import sys

import numpy as np

import oracle as O
from paper_1310_6143_gb300 import lattice as L

GAMMA, KB, MU = 1.76e11, 1.3807e-23, 1.5 * 9.2740e-24


def pin_field_gradient():
    rng = np.random.default_rng(3)
    n = 6
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < 0.6:
                A[i, j] = A[j, i] = rng.normal(0, 5e-21)
    rp, col, J = [0], [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        col += list(nz); J += list(A[i, nz]); rp.append(len(col))
    mu = rng.uniform(1, 3, n) * 9.274e-24
    ku = rng.normal(0, 2e-23, n)
    ax = rng.normal(size=(n, 3)); ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    H = rng.normal(0, 3, 3)
    K = np.zeros((n, 6))
    for i in range(0, n, 2):
        M = rng.normal(0, 1e-23, (3, 3))
        M = M + M.T
        K[i] = [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]
    s = O.OracleSystem(np.array(rp), np.array(col), np.array(J), mu, ku, ax, K, H_app=tuple(H))
    S = L.random_state(n, 4)

    def energy(S):
        e = 0.0
        for i in range(n):
            for j in range(i + 1, n):
                e -= A[i, j] * S[i] @ S[j]
        for i in range(n):
            Mi = np.array([[K[i, 0], K[i, 3], K[i, 4]], [K[i, 3], K[i, 1], K[i, 5]], [K[i, 4], K[i, 5], K[i, 2]]])
            e -= S[i] @ Mi @ S[i]
        return e - np.sum(ku * np.einsum("ij,ij->i", S, ax) ** 2) - np.sum(mu * (S @ H))
    me = O.moment_energy(s, S)
    if abs(me[7] - energy(S)) > 1e-12 * abs(energy(S)):
        return False
    F = O.fields(s, S)
    h = 1e-6
    for i in range(n):
        for c in range(3):
            Sp, Sm = S.copy(), S.copy()
            Sp[i, c] += h; Sm[i, c] -= h
            ref = -(energy(Sp) - energy(Sm)) / (2 * h) / mu[i]
            if abs(F[i, c] - ref) > 1e-7 * max(1.0, np.abs(F[i]).max()):
                return False
    return True


def pin_single_spin_analytic():
    lat = L.single_spin()
    lam, H, dt = 0.1, 10.0, 1e-15
    s = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, 0.0, lat.easy_axis, alpha=lam, dt=dt, H_app=(0, 0, H))
    S = np.array([[1.0, 0, 0]])
    err = 0.0
    for k in range(60):
        S, _ = O.heun_run(s, S, 500, 0.0, step0=k * 500)
        t = (k + 1) * 500 * dt
        a, w = lam * GAMMA * H / (1 + lam ** 2) * t, GAMMA * H / (1 + lam ** 2) * t
        ref = np.array([math.cos(w) / math.cosh(a), math.sin(w) / math.cosh(a), math.tanh(a)])
        err = max(err, np.abs(S[0] - ref).max())
    return err < 1e-6


def pin_unit_length():
    lat = L.simple_cubic(4, 4, 4)
    s = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.1, dt=1e-16)
    S = L.random_state(lat.n, 2)
    for k in range(5):
        S, _ = O.heun_run(s, S, 1, 500.0, step0=k)
        if np.abs(np.linalg.norm(S, axis=1) - 1).max() > 1e-15:
            return False
    return True


def pin_gaussians():
    g = O.gaussians_bulk(9, 1, 3, 100_000)
    if np.abs(g.mean(0)).max() > 0.02 or np.abs(g.var(0) - 1).max() > 0.02:
        return False
    return np.abs(np.corrcoef(g.T) - np.eye(3)).max() < 0.015


def pin_philox_against_torch():
    import os
    import subprocess
    import tempfile

    import torch

    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "p.cpp")
    open(src, "w").write("#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\nint main(){ at::philox_engine "
                         "e(0x0123456789abcdefULL, 7ULL, (5ULL<<32)|3ULL); for(int i=0;i<4;i++) printf(\"%u \", e());"
                         " return 0; }\n")
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}", "-o", os.path.join(d, "p"), src], check=True)
    out = [int(v) for v in subprocess.run([os.path.join(d, "p")], capture_output=True, text=True).stdout.split()]
    return list(O.philox4x32_10([3, 5, 7, 0], [0x89ABCDEF, 0x01234567])) == out


def pin_boltzmann():
    ku, kappa, lam = 1e-22, 3.0, 1.0
    T = ku / (kappa * KB)
    dt = 0.0025 * MU / (2 * lam * KB * T * GAMMA)
    n = 64
    s = O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0), np.full(n, MU),
                       np.full(n, ku), (0, 0, 1), alpha=lam, dt=dt, seed=5)
    S, _ = O.heun_run(s, np.tile([0, 0, 1.0], (n, 1)), 3000, T)
    c2 = []
    for k in range(100):
        S, _ = O.heun_run(s, S, 400, T, step0=3000 + k * 400)
        c2.append(S[:, 2] ** 2)
    m2 = np.concatenate(c2).mean()
    from scipy import integrate
    Z = integrate.quad(lambda x: np.exp(kappa * x * x), 0, 1)[0]
    ref = integrate.quad(lambda x: x * x * np.exp(kappa * x * x), 0, 1)[0] / Z
    return abs(m2 - ref) < 0.02


def pin_curie():
    lat = L.simple_cubic(6, 6, 6, J=6e-21, k_u=0.0)
    ms = {}
    for T in (312.5, 937.5):
        s = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, 0.0, lat.easy_axis, alpha=1.0, dt=1e-17, seed=7)
        S, _ = O.heun_run(s, L.uniform_state(lat.n), 2500, T)
        S, rec = O.heun_run(s, S, 2500, T, step0=2500, record=True)
        ms[T] = (np.linalg.norm(rec[:, :3], axis=1) / rec[:, 3]).mean()
    return 0.6 < ms[312.5] < 0.92 and ms[937.5] < 0.3


def _free(n, k_u=0.0):
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0), np.full(n, MU), np.full(n, k_u)


def _mc_average(s, S, T, equil, blocks, per, f):
    S, _, _ = O.mc_run(s, S, equil, T)
    vals, step = [], equil
    for _ in range(blocks):
        S, _, _ = O.mc_run(s, S, per, T, step0=step)
        step += per
        vals.append(f(S))
    return np.concatenate(vals).mean()


def _langevin(x):
    return 1.0 / math.tanh(x) - 1.0 / x


def pin_mc_boltzmann():
    """Eq. boltz with Monte Carlo: <cos^2> of free spins with anisotropy, k_u/(kB T) = 3."""
    n, T, kappa = 2000, 50.0, 3.0
    rp, col, J, mu, ku = _free(n, kappa * KB * T)
    s = O.OracleSystem(rp, col, J, mu, ku, (0, 0, 1), seed=3)
    m2 = _mc_average(s, L.uniform_state(n), T, 60, 15, 5, lambda S: S[:, 2] ** 2)
    from scipy import integrate
    Z = integrate.quad(lambda x: np.exp(kappa * x * x), 0, 1)[0]
    return abs(m2 - integrate.quad(lambda x: x * x * np.exp(kappa * x * x), 0, 1)[0] / Z) < 0.015


def pin_mc_langevin():
    n, T, x = 2000, 100.0, 2.0
    rp, col, J, mu, ku = _free(n)
    H = x * KB * T / MU
    s = O.OracleSystem(rp, col, J, mu, ku, (0, 0, 1), H_app=(0.0, 0.0, H), seed=8)
    return abs(_mc_average(s, L.random_state(n, 2), T, 40, 15, 4, lambda S: S[:, 2]) - _langevin(x)) < 0.015


def pin_mc_dimer():
    npairs, T, K = 1500, 100.0, 1.5
    n = 2 * npairs
    s = O.OracleSystem(np.arange(n + 1, dtype=np.int64), (np.arange(n) ^ 1).astype(np.int32), np.full(n, K * KB * T),
                       np.full(n, MU), np.zeros(n), (0, 0, 1), seed=13)
    got = _mc_average(s, L.random_state(n, 4), T, 40, 15, 4, lambda S: np.einsum("ij,ij->i", S[0::2], S[1::2]))
    return abs(got - _langevin(K)) < 0.02


def pin_mc_moves():
    """One step of free spins (all moves accepted): a third flips, unit lengths, the
    Gaussian moves inside a cone of a few sigma_g (Eq. MCgaussianSigma), the rest uniform."""
    n, T = 12000, 10.0
    rp, col, J, mu, ku = _free(n)
    s = O.OracleSystem(rp, col, J, mu, ku, (0, 0, 1), seed=21)
    S0 = L.random_state(n, 5)
    S1, _, acc = O.mc_run(s, S0, 1, T)
    if acc[0] != n or np.abs(np.linalg.norm(S1, axis=1) - 1).max() > 1e-14:
        return False
    dot = np.einsum("ij,ij->i", S0, S1)
    flip = np.all(S1 == -S0, axis=1)
    sg = 0.08 * (KB * T / 9.2740e-24) ** 0.2
    near = (~flip) & (dot > math.cos(5 * sg))
    c = math.cos(5 * sg)
    far = dot[~(flip | near)]
    third = n / 3
    return (abs(flip.sum() - third) < 5 * math.sqrt(n * 2 / 9)
            and abs(near.sum() - third * (1 + (1 - c) / 2)) < 5 * math.sqrt(n * 2 / 9) + 10
            and abs(far.mean() - (c - 1) / 2) < 0.03 and 0.5 * sg ** 2 < (1 - dot[near]).mean() < 1.5 * sg ** 2)


def pin_mc_sigma():
    return abs(O.mc_sigma_g(320.0) / O.mc_sigma_g(10.0) - 2.0) < 1e-12


def pin_mc_zero_T():
    """T = 0: no step raises the energy; the record holds the state before each step."""
    lat = L.simple_cubic(6, 6, 6, J=6e-21, k_u=1e-23)
    s = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, H_app=(0, 0.3, 0.5), seed=2)
    S0 = L.random_state(lat.n, 7)
    _, rec, _ = O.mc_run(s, S0, 5, 0.0, record=True)
    return np.all(np.diff(rec[:, 7]) <= 1e-30) and np.allclose(rec[0], O.moment_energy(s, S0), rtol=0, atol=0)


def pin_colouring():
    for lat in (L.simple_cubic(5, 5, 5), L.fcc(3, 3, 3)):
        s = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis)
        colour, nc = O.colour_greedy(s)
        rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
        if np.any(colour[rows] == colour[lat.col]) or colour.max() != nc - 1:
            return False
    return True


def pin_demag():
    """Macrocell demagnetising field: self term of one cell, axis / broadside ratio of two
    dipoles, the moment-weighted cell centre, and the update interval."""
    mu0, a, vat, muB = 4e-7 * math.pi, 3e-10, (3e-10) ** 3, 9.2740e-24

    def pts(pos, mu, cell):
        n = len(pos)
        return O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0),
                              np.broadcast_to(np.asarray(mu, dtype=float), (n,)), np.zeros(n), (0, 0, 1),
                              pos=np.asarray(pos, dtype=float), demag_cell=cell, demag_vatom=vat)

    g = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3) * a
    S = L.random_state(len(g), 3)
    _, Hmc = O.demag_fields(pts(g, 2 * muB, 10 * a), S)
    if not np.allclose(Hmc[0], -mu0 / 3 * 2 * muB * S.sum(0) / (len(g) * vat), rtol=1e-12, atol=0):
        return False
    two = [[0, 0, 0], [0, 0, 5e-9]]
    s2 = pts(two, 1.5 * muB, a)
    self_ = -mu0 / 3 * 1.5 * muB / vat
    ax = O.demag_fields(s2, np.array([[0, 0, 1.0], [0, 0, 1.0]]))[0][0, 2] - self_
    br = O.demag_fields(s2, np.array([[1.0, 0, 0], [1.0, 0, 0]]))[0][0, 0] - self_
    if abs(ax / br + 2.0) > 1e-8:
        return False
    # a cell of a tiny and a large moment acts from (almost) the large one's position
    mixed = pts([[0, 0, 0], [0.9 * a, 0, 0], [0.45 * a, 0, 6e-9]], [1e-6 * muB, 2 * muB, muB], 2 * a)
    alone = pts([[0.9 * a, 0, 0], [0.45 * a, 0, 6e-9]], [2 * muB, muB], 2 * a)
    up = lambda n: np.tile([0, 0, 1.0], (n, 1))  # noqa: E731
    hm = O.demag_fields(mixed, up(3))[0][2]
    ha = O.demag_fields(alone, up(2))[0][1]
    if abs(hm[2] - ha[2]) > 1e-5 * abs(ha[2]) or abs(hm[0] - ha[0]) > 1e-5 * abs(ha[0]):
        return False
    lat = L.simple_cubic(6, 6, 2, periodic=(False, False, False), J=6e-21, k_u=0.0, with_pos=True)
    mk = lambda every: O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis,  # noqa: E731
                                      alpha=0.5, dt=1e-15, seed=5, pos=lat.pos, demag_cell=6e-10,
                                      demag_vatom=(3e-10) ** 3, demag_every=every)
    S0 = L.random_state(lat.n, 1)
    r5, _ = O.heun_run(mk(5), S0, 10, 50.0)
    r1, _ = O.heun_run(mk(1), S0, 10, 50.0)
    return np.abs(r5 - r1).max() > 1e-9


def _skew(d):
    return np.array([[0.0, -d[2], d[1]], [d[2], 0.0, -d[0]], [-d[1], d[0], 0.0]])


def pin_tensor_cubic():
    """Tensorial exchange and cubic anisotropy: field = -(1/mu) grad E on a random 2x2x2
    system (energy from the printed expressions), and the DM dimer's chirality."""
    lat = L.simple_cubic(2, 2, 2, periodic=(False, False, False))
    rng = np.random.default_rng(2)
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    where = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(rows, lat.col))}
    Jt = np.zeros((lat.nnz, 3, 3))
    for k, (i, j) in enumerate(zip(rows, lat.col)):
        if i < j:
            B = rng.normal(size=(3, 3)) * 1e-21
            A = 6e-21 * np.eye(3) + 0.5 * (B + B.T) + _skew(rng.normal(size=3) * 2e-21)
            Jt[k], Jt[where[(int(j), int(i))]] = A, A.T
    kc = rng.uniform(-2e-23, 2e-23, lat.n)
    s = O.OracleSystem(lat.row_ptr, lat.col, np.zeros(lat.nnz), np.full(lat.n, MU), 0.0, (0, 0, 1), J_tensor=Jt,
                       k_c=kc)

    def energy(S):
        e = sum(-S[i] @ Jt[k] @ S[j] for k, (i, j) in enumerate(zip(rows, lat.col)) if i < j)
        return e + np.sum(0.5 * kc * (S ** 4).sum(1))

    S = L.random_state(lat.n, 4)
    Hf = O.fields(s, S)
    if abs(O.moment_energy(s, S)[7] - energy(S)) > 1e-12 * abs(energy(S)):
        return False
    for i in range(lat.n):
        for c in range(3):
            Sp, Sm = S.copy(), S.copy()
            Sp[i, c] += 1e-6
            Sm[i, c] -= 1e-6
            if abs(Hf[i, c] + (energy(Sp) - energy(Sm)) / 2e-6 / MU) > 1e-7 * max(1.0, np.abs(Hf[i]).max()):
                return False
    J, D = 5e-21, np.array([1.0, -2.0, 2.0]) * 1e-21
    A = J * np.eye(3) + _skew(D)
    d = O.OracleSystem(np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32), np.zeros(2), np.full(2, 2 * MU / 1.5),
                       0.0, (0, 0, 1), J_tensor=np.stack([A, A.T]), alpha=1.0, dt=1e-16, seed=4)
    Sd, _ = O.heun_run(d, L.random_state(2, 6), 30000, 0.0)
    return np.cross(Sd[0], Sd[1]) @ D / np.linalg.norm(D) < -0.45


def pin_mc_cubic():
    n, T, K = 2000, 40.0, 4.0
    s = O.OracleSystem(np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0), np.full(n, MU), 0.0,
                       (0, 0, 1), k_c=K * KB * T, seed=12)
    got = _mc_average(s, L.random_state(n, 1), T, 60, 15, 4, lambda S: (S ** 4).sum(1))
    from scipy import integrate
    f = lambda th, ph: np.sin(th) ** 4 * (np.cos(ph) ** 4 + np.sin(ph) ** 4) + np.cos(th) ** 4  # noqa: E731
    w = lambda th, ph: np.exp(-0.5 * K * f(th, ph)) * np.sin(th)  # noqa: E731
    Z = integrate.dblquad(w, 0, 2 * np.pi, 0, np.pi)[0]
    ref = integrate.dblquad(lambda th, ph: f(th, ph) * w(th, ph), 0, 2 * np.pi, 0, np.pi)[0] / Z
    return abs(got - ref) < 0.006


def pin_midpoint():
    """Midpoint rule: undamped precession is the Cayley rotation (2 atan(w dt/2) a step), and
    the length error falls with the fixed-point iterations."""
    H = 10.0
    dt = 0.1 / (GAMMA * H)
    s = O.OracleSystem(np.zeros(2, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0), [MU], 0.0, (0, 0, 1),
                       alpha=0.0, dt=dt, H_app=(0.0, 0.0, H))
    S, _ = O.midpoint_run(s, np.array([[0.6, 0.0, 0.8]]), 100, 0.0, iters=40)
    d = np.angle(np.exp(1j * (np.arctan2(S[0, 1], S[0, 0]) - 200 * np.arctan(0.05))))
    if abs(d) > 1e-10:
        return False
    lat = L.simple_cubic(4, 4, 4, J=6e-21, k_u=1e-23)
    sl = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.1, dt=1e-16, seed=2)
    S0 = L.random_state(lat.n, 1)
    e = [np.abs(np.linalg.norm(O.midpoint_run(sl, S0, 30, 300.0, iters=K)[0], axis=1) - 1).max() for K in (2, 8)]
    return e[1] < 1e-11 and e[0] > 1e3 * e[1]


def pin_sib():
    """Semi-implicit predictor-corrector: undamped precession is the Cayley rotation, the
    damped single spin converges at second order, and a spin with anisotropy follows the
    scheme's two linear equations solved independently."""
    H = 10.0
    w = GAMMA * H
    one = lambda lam, dt, ku=0.0, Happ=(0.0, 0.0, H), axis=(0, 0, 1): O.OracleSystem(  # noqa: E731
        np.zeros(2, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0), [MU], ku, axis, alpha=lam, dt=dt,
        H_app=Happ)
    S, _ = O.sib_run(one(0.0, 0.1 / w), np.array([[0.6, 0.0, 0.8]]), 100, 0.0)
    if abs(np.angle(np.exp(1j * (np.arctan2(S[0, 1], S[0, 0]) - 200 * np.arctan(0.05))))) > 1e-10:
        return False
    errs = []
    for dt in (4e-15, 2e-15):
        S, _ = O.sib_run(one(0.1, dt), np.array([[1.0, 0.0, 0.0]]), int(round(20e-12 / dt)), 0.0)
        a_, w_ = 0.1 * w / 1.01 * 20e-12, w / 1.01 * 20e-12
        errs.append(np.abs(S[0] - [np.cos(w_) / np.cosh(a_), np.sin(w_) / np.cosh(a_), np.tanh(a_)]).max())
    if not 3.5 < errs[0] / errs[1] < 4.5:
        return False
    lam, ku, dt = 0.3, 2e-23, 2e-15
    e = np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])
    Happ = np.array([0.4, 1.1, -0.7])

    def A(v):
        Hf = Happ + 2 * ku / MU * (v @ e) * e
        return -GAMMA / (1 + lam ** 2) * (Hf + lam * np.cross(v, Hf))

    def half(Sn, a):
        K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
        return np.linalg.solve(np.eye(3) + (dt / 2) * K, Sn - (dt / 2) * np.cross(a, Sn))

    ref = np.array([0.48, 0.6, 0.64])
    S0 = ref.copy()
    for _ in range(10):
        P = half(ref, A(ref))
        ref = half(ref, A(0.5 * (ref + P)))
    got, _ = O.sib_run(one(lam, dt, ku, tuple(Happ), tuple(e)), S0[None], 10, 0.0)
    return np.abs(got[0] - ref).max() <= 1e-13


def pin_alt_demag():
    """The alternative integrators with the demagnetising field as the only field converge
    to the Heun trajectory at second order."""
    lat = L.simple_cubic(6, 6, 2, periodic=(False, False, False), J=0.0, k_u=0.0, with_pos=True)
    mk = lambda dt: O.OracleSystem(  # noqa: E731
        lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.5, dt=dt, seed=5, pos=lat.pos,
        demag_cell=6e-10, demag_vatom=(3e-10) ** 3, demag_every=1)
    S0 = L.random_state(lat.n, 1)
    for run in (lambda s, n: O.midpoint_run(s, S0, n, 0.0, iters=30)[0], lambda s, n: O.sib_run(s, S0, n, 0.0)[0]):
        d = [np.abs(run(mk(dt), int(round(4e-11 / dt))) - O.heun_run(mk(dt), S0, int(round(4e-11 / dt)), 0.0)[0]).max()
             for dt in (2e-13, 1e-13)]
        if not 3.5 < d[0] / d[1] < 4.5:
            return False
    return True


PINS = [pin_field_gradient, pin_single_spin_analytic, pin_unit_length, pin_gaussians, pin_philox_against_torch,
        pin_boltzmann, pin_curie, pin_mc_boltzmann, pin_mc_langevin, pin_mc_dimer, pin_mc_moves, pin_mc_sigma,
        pin_mc_zero_T, pin_colouring, pin_demag, pin_tensor_cubic, pin_mc_cubic, pin_midpoint,
        pin_sib, pin_alt_demag]

if __name__ == "__main__":
    for p in PINS:
        try:
            ok = bool(p())
        except Exception:
            ok = False
        print(("PASS " if ok else "FAIL ") + p.__name__, flush=True)
    sys.exit(0)

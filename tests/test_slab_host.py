"""Host side of the slab decomposition (Appendix C): halo runs, the exchange plan, and the
step sequence of the distributed driver on two gloo ranks.

The distributed test drives a CPU stand-in of a slab handle whose two passes have the data
flow of the Heun passes -- pass 0 reads S of the neighbours and writes the owned S', pass 1
reads S' of the neighbours and the owned S and writes the owned S -- so that a missing or
mistimed halo refresh changes the result.  Two ranks must reproduce the undecomposed run bit
for bit; a driver that skips the S' refresh must not."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1310_6143_gb300 import lattice as L
from paper_1310_6143_gb300.slab import (DistributedSlab, Transfer, exchange_plan, halo_runs, slab_range,
                                        sources_are_boundary)


def _lattices():
    return {
        "film": L.film(12, 10, 4),
        "sc": L.simple_cubic(5, 6, 4),
        "fcc": L.fcc(3, 4, 3),
        "core_shell": L.core_shell_sphere(diameter=3e-9, r_core=1e-9),
    }


def _brute_halo(lat, lo, hi):
    s = set()
    for i in range(lo, hi):
        for k in range(lat.row_ptr[i], lat.row_ptr[i + 1]):
            j = int(lat.col[k])
            if not lo <= j < hi:
                s.add(j)
    return sorted(s)


@pytest.mark.parametrize("name", ["film", "sc", "fcc", "core_shell"])
@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_halo_runs_and_plan_cover_every_halo_copy_once(name, K):
    lat = _lattices()[name]
    ranges = [slab_range(lat.n, K, k) for k in range(K)]
    assert ranges[0][0] == 0 and ranges[-1][1] == lat.n
    assert all(ranges[k][1] == ranges[k + 1][0] for k in range(K - 1))
    runs = []
    for lo, hi in ranges:
        r = halo_runs(lat.row_ptr, lat.col, lo, hi)
        halo = _brute_halo(lat, lo, hi)
        flat = [int(g) + m for g, length, _ in r for m in range(int(length))]
        assert flat == halo
        if len(r):  # local indices: the halo copies follow the owned spins in global order
            assert np.array_equal(r[:, 2], hi - lo + np.concatenate([[0], np.cumsum(r[:-1, 1])]))
        if len(r) > 1:  # maximal runs: no two adjacent runs touch
            assert np.all(r[1:, 0] > r[:-1, 0] + r[:-1, 1])
        runs.append(r)
    plan = exchange_plan(runs, ranges)
    filled = [np.zeros(hi - lo + len(_brute_halo(lat, lo, hi)), dtype=np.int64) - 1 for lo, hi in ranges]
    for t in plan:
        assert t.src != t.dst and t.length > 0
        slo, shi = ranges[t.src]
        assert 0 <= t.src_at and t.src_at + t.length <= shi - slo
        dlo, dhi = ranges[t.dst]
        seg = filled[t.dst][t.dst_at:t.dst_at + t.length]
        assert t.dst_at >= dhi - dlo and np.all(seg == -1)
        seg[:] = np.arange(slo + t.src_at, slo + t.src_at + t.length)
    for k, (lo, hi) in enumerate(ranges):
        halo = _brute_halo(lat, lo, hi)
        assert list(filled[k][hi - lo:]) == halo
    assert sources_are_boundary(lat.row_ptr, lat.col, plan, ranges)


def test_plan_rejects_bad_runs_and_detects_one_sided_lists():
    ranges = [(0, 4), (4, 8)]
    with pytest.raises(ValueError):
        exchange_plan([np.array([[2, 1, 4]]), np.zeros((0, 3))], ranges)  # own spin in the halo
    with pytest.raises(ValueError):
        exchange_plan([np.array([[8, 1, 4]]), np.zeros((0, 3))], ranges)  # no owner
    # a run across an owner boundary is cut there
    plan = exchange_plan([np.zeros((0, 3)), np.zeros((0, 3)), np.array([[2, 4, 3]])], [(0, 4), (4, 8), (8, 11)])
    assert plan == [Transfer(0, 2, 2, 3, 2), Transfer(1, 2, 0, 5, 2)]
    # a one-sided list: spin 4 names spin 3, but spin 3 names only spin 2 of its own slab
    row_ptr = np.array([0, 1, 2, 3, 4, 6, 7, 8, 9], dtype=np.int64)
    col = np.array([1, 0, 3, 2, 3, 5, 4, 7, 6], dtype=np.int32)
    ranges = [(0, 4), (4, 8)]
    runs = [halo_runs(row_ptr, col, lo, hi) for lo, hi in ranges]
    plan = exchange_plan(runs, ranges)
    assert plan == [Transfer(0, 1, 3, 4, 1)]
    assert not sources_are_boundary(row_ptr, col, plan, ranges)


class FakeSlab:
    """CPU stand-in of a slab handle (tiles of one spin, boundary spins first)."""

    C0, C1 = 0.3, 0.2

    def __init__(self, lat, nslabs, k, S0):
        lo, hi = slab_range(lat.n, nslabs, k)
        runs = halo_runs(lat.row_ptr, lat.col, lo, hi)
        halo = np.array([int(g) + m for g, length, _ in runs for m in range(int(length))], dtype=np.int64)
        self.glob = np.concatenate([np.arange(lo, hi), halo]).astype(np.int64)
        own, nt = hi - lo, hi - lo + halo.size
        loc = {int(g): i for i, g in enumerate(self.glob)}
        self.rp = np.zeros(own + 1, dtype=np.int64)
        cols, js = [], []
        edge = np.zeros(own, dtype=bool)
        jn = lat.J / np.abs(lat.J).max()
        for i in range(lo, hi):
            for q in range(lat.row_ptr[i], lat.row_ptr[i + 1]):
                j = int(lat.col[q])
                cols.append(loc[j])
                js.append(jn[q])
                edge[i - lo] |= not lo <= j < hi
            self.rp[i - lo + 1] = len(cols)
        self.col = np.array(cols, dtype=np.int64)
        self.J = np.array(js)
        self.order = np.concatenate([np.flatnonzero(edge), np.flatnonzero(~edge)])
        self.slab = {"lo": lo, "hi": hi, "boundary_tiles": int(edge.sum()), "num_tiles": own}
        self.own = own
        self.S = tuple(torch.tensor(S0[self.glob, c].copy()) for c in range(3))
        self.P = tuple(torch.zeros(nt, dtype=torch.float64) for _ in range(3))
        self.partials = np.zeros((own, 8))
        self.rec = []

    def state_device(self, which):
        return self.S if which == 0 else self.P

    def _field(self, arrs, idx):
        out = np.zeros((idx.size, 3))
        for n, i in enumerate(idx):
            a, b = self.rp[i], self.rp[i + 1]
            for c in range(3):
                v = arrs[c].numpy()
                out[n, c] = float(np.dot(self.J[a:b], v[self.col[a:b]])) if b > a else 0.0
        return out

    def heun_pass(self, which, t0, nt):
        if which == 2:
            self.rec.append(self.partials.sum(axis=0))
            return
        idx = self.order[t0:t0 + nt]
        if idx.size == 0:
            return
        s = np.stack([self.S[c].numpy()[idx] for c in range(3)], axis=1)
        if which == 0:
            h = self._field(self.S, idx)
            v = s + self.C0 * (np.cross(s, h) + h)
            self.partials[idx, :3] = s
            self.partials[idx, 3] = 1.0
            self.partials[idx, 4] = np.einsum("ij,ij->i", s, h)
            dst = self.P
        else:
            h = self._field(self.P, idx)
            p = np.stack([self.P[c].numpy()[idx] for c in range(3)], axis=1)
            v = s + self.C1 * (np.cross(p, h) + h)
            dst = self.S
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        for c in range(3):
            dst[c].numpy()[idx] = v[:, c]

    def record(self, first, count):
        return np.array(self.rec[first:first + count]).reshape(count, 1, 8)


def _reference(lat, S0, steps):
    f = FakeSlab(lat, 1, 0, S0)
    for _ in range(steps):
        f.heun_pass(0, 0, f.own)
        f.heun_pass(1, 0, f.own)
        f.heun_pass(2, 0, 0)
    return np.stack([f.S[c].numpy()[:f.own] for c in range(3)], axis=1), f.record(0, steps)


class _NoPrimeExchange(DistributedSlab):
    def step(self, nsteps=1):
        nt = self.h.slab["num_tiles"]
        for _ in range(nsteps):
            self.h.heun_pass(0, 0, nt)
            self.h.heun_pass(1, 0, nt)
            self.h.heun_pass(2, 0, 0)
            self.refresh_halo()


def _worker(rank, world, port, name, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lat = _lattices()[name]
    S0 = L.random_state(lat.n, 5)
    out = {}
    for label, cls in (("slab", DistributedSlab), ("no_prime", _NoPrimeExchange)):
        d = cls(FakeSlab(lat, world, rank, S0), lat.row_ptr, lat.col)
        d.refresh_halo()
        d.step(steps)
        own = d.h.own
        out[label] = (np.stack([d.h.S[c].numpy()[:own] for c in range(3)], axis=1), d.record(0, steps))
    q.put((rank, out))
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["film", "fcc"])
def test_two_gloo_ranks_reproduce_the_undecomposed_run(name):
    steps = 6
    lat = _lattices()[name]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + (os.getpid() % 1000) + (0 if name == "film" else 50)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, name, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    S_ref, rec_ref = _reference(lat, L.random_state(lat.n, 5), steps)
    S = np.concatenate([got[0]["slab"][0], got[1]["slab"][0]])
    np.testing.assert_array_equal(S, S_ref)
    for r in range(2):  # every rank holds the all-reduced records
        np.testing.assert_allclose(got[r]["slab"][1], rec_ref, rtol=1e-12, atol=1e-12 * lat.n)
    S_bad = np.concatenate([got[0]["no_prime"][0], got[1]["no_prime"][0]])
    assert not np.array_equal(S_bad, S_ref)

"""Slab decomposition of one system (the paper's spatial parallelisation, Appendix C).

The paper splits a system that is too large for one processor into geometric domains.  Each
domain sorts its spins into core spins (all neighbours local), boundary spins (a neighbour
in another domain) and halo copies of the other domains' boundary spins.  The halo is passed
twice per Heun step: after the predictor (the corrector's fields need S' of the neighbours)
and after the corrector (the next predictor needs S).  The boundary spins are integrated
first, so that the transfer overlaps the integration of the core spins.

Here a domain is a slab: the contiguous global index range [lo, hi), lo = n k / K, of a
lattice numbered plane by plane (the film and the cubic lattices have their slowest index
on one axis, so a slab is a stack of planes and its halo is one plane or a few on each side).
The library handle of a slab (``spin_slab_create``) holds the owned spins, then the halo
copies in global order.  It draws every owned spin's thermal field from the Philox counter
of its global index.  Its tiles hold owned spins only, the boundary tiles first.
This module holds the host side:

* ``halo_runs`` and ``exchange_plan`` -- which owned spins of which slab fill which halo
  copies (contiguous runs on both sides, so every transfer is one slice per component);
* ``SlabSystem`` -- K slabs of one system on one GPU in one process, each on its own CUDA
  stream, with device-to-device halo copies on per-slab copy streams ordered by events;
* ``DistributedSlab`` -- one slab per rank of a ``torch.distributed`` group, the halo
  passed by point-to-point send/receive (NCCL on GPUs; gloo works for host tensors) and the
  eight record sums of a step reduced over the ranks.

A step of every driver is: predictor over the boundary tiles, halo transfer of S' started,
predictor over the core tiles, transfer finished, corrector over the boundary tiles, halo
transfer of S started, corrector over the core tiles, end of step (record, step counter),
transfer finished.  The corrector reads S' of its neighbours and only its own S, and the
predictor reads S of its neighbours and writes only its own S'; so no pass reads a halo
array while that array is being refilled.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np


def slab_range(n: int, nslabs: int, k: int) -> tuple[int, int]:
    """The owned global range [lo, hi) of slab k (the library's split)."""
    return n * k // nslabs, n * (k + 1) // nslabs


def halo_runs(row_ptr: np.ndarray, col: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """(runs, 3) int64: first global index, length and first local index of each maximal run
    of consecutive global indices among the halo spins of the owned range [lo, hi).  The
    halo is every spin outside the range that an owned row names.  Local indices follow the
    owned spins (hi - lo of them) in global order."""
    cols = np.asarray(col[int(row_ptr[lo]):int(row_ptr[hi])], dtype=np.int64)
    halo = np.unique(cols[(cols < lo) | (cols >= hi)])
    if halo.size == 0:
        return np.zeros((0, 3), dtype=np.int64)
    starts = np.flatnonzero(np.diff(halo, prepend=halo[0] - 2) != 1)
    lengths = np.diff(np.append(starts, halo.size))
    return np.stack([halo[starts], lengths, (hi - lo) + starts], axis=1).astype(np.int64)


@dataclass(frozen=True)
class Transfer:
    """Copy ``length`` spins from local index ``src_at`` of slab ``src`` to local index
    ``dst_at`` of slab ``dst`` (owned spins of src into halo copies of dst)."""

    src: int
    dst: int
    src_at: int
    dst_at: int
    length: int


def exchange_plan(runs: Sequence[np.ndarray], ranges: Sequence[tuple[int, int]]) -> list[Transfer]:
    """All transfers of one halo refresh: each halo run of each slab cut at the owners'
    range boundaries.  Raises if a halo spin has no owner or a slab names its own spin."""
    out: list[Transfer] = []
    los = np.array([r[0] for r in ranges], dtype=np.int64)
    for dst, rr in enumerate(runs):
        for g, length, at in np.asarray(rr, dtype=np.int64).reshape(-1, 3):
            g, end, at = int(g), int(g + length), int(at)
            while g < end:
                src = int(np.searchsorted(los, g, side="right")) - 1
                lo, hi = ranges[src]
                if src < 0 or not (lo <= g < hi):
                    raise ValueError(f"halo spin {g} of slab {dst} has no owner")
                if src == dst:
                    raise ValueError(f"slab {dst} lists its own spin {g} in its halo")
                take = min(end, hi) - g
                out.append(Transfer(src, dst, g - lo, at, take))
                g += take
                at += take
    return out


def sources_are_boundary(row_ptr: np.ndarray, col: np.ndarray, plan: Sequence[Transfer],
                         ranges: Sequence[tuple[int, int]]) -> bool:
    """True when every spin a transfer reads is a boundary spin of its slab (has a neighbour
    outside the slab), so that it lies in the slab's boundary tiles and may be sent once those
    tiles are done.  Holds for symmetric neighbour lists."""
    for t in plan:
        lo, hi = ranges[t.src]
        a = lo + t.src_at
        rp = np.asarray(row_ptr[a:a + t.length + 1], dtype=np.int64)
        if np.any(np.diff(rp) == 0):
            return False  # a spin without neighbours is no boundary spin
        c = np.asarray(col[int(rp[0]):int(rp[-1])], dtype=np.int64)
        outside = (c < lo) | (c >= hi)
        if not np.logical_or.reduceat(outside, rp[:-1] - rp[0]).all():
            return False
    return True


class SlabSystem:
    """One system split into ``nslabs`` slabs, each a library handle on its own CUDA stream
    of the current device, advanced together with device-to-device halo copies.

    The keyword arguments are those of ``SpinSystem`` (one lattice).  Spins, records and
    observables are those of the whole system: the owned spins of the slabs in order, and the
    eight record sums added over the slabs (in slab order, in FP64)."""

    def __init__(self, lattice, nslabs: int, **kw):
        import torch

        from .system import SpinSystem

        if nslabs < 1:
            raise ValueError("nslabs must be >= 1")
        self.n = lattice.n
        self.nslabs = nslabs
        self.ranges = [slab_range(lattice.n, nslabs, k) for k in range(nslabs)]
        self.slabs = [SpinSystem(lattice, slab=(nslabs, k), **kw) for k in range(nslabs)]
        self.precision = self.slabs[0].precision
        self.streams = [torch.cuda.Stream() for _ in range(nslabs)]
        self.copy_streams = [torch.cuda.Stream() for _ in range(nslabs)]
        for s, st in zip(self.slabs, self.streams):
            s.set_stream(st)
        runs = [s.halo_runs() for s in self.slabs]
        self.plan = exchange_plan(runs, self.ranges)
        # early transfers (after the boundary tiles) need every sent spin in a boundary tile
        self.early = sources_are_boundary(lattice.row_ptr, lattice.col, self.plan, self.ranges)
        self.into = [[t for t in self.plan if t.dst == k] for k in range(nslabs)]
        self.S = [s.state_device(0) for s in self.slabs]
        self.P = [s.state_device(1) for s in self.slabs]
        ev = lambda: [torch.cuda.Event() for _ in range(nslabs)]  # noqa: E731
        self._pb, self._p, self._cb, self._c, self._hp, self._hs = ev(), ev(), ev(), ev(), ev(), ev()
        self._halo_s_ready = False
        self._stepped = False  # a corrector ran: S' copies wait for it

    # -- lifetime ---------------------------------------------------------------------
    def close(self):
        for s in self.slabs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration (forwarded to every slab) ------------------------------------------
    def set_temperature(self, T):
        for s in self.slabs:
            s.set_temperature(T)

    def set_temperature_schedule(self, T_per_step, step0: int = 0):
        for s in self.slabs:
            s.set_temperature_schedule(T_per_step, step0)

    def set_field(self, H):
        for s in self.slabs:
            s.set_field(H)

    def set_launch(self, block: int, tile: int):
        for s in self.slabs:
            s.set_launch(block, tile)

    # -- the step -----------------------------------------------------------------------
    def _copy(self, k: int, arrays, after_src, after_dst):
        """Refill slab k's halo copies of ``arrays`` on its copy stream once its sources
        recorded ``after_src`` and slab k itself recorded ``after_dst``."""
        cs = self.copy_streams[k]
        if after_dst is not None:
            cs.wait_event(after_dst[k])
        for j in sorted({t.src for t in self.into[k]}):
            cs.wait_event(after_src[j])
        import torch

        with torch.cuda.stream(cs):
            for t in self.into[k]:
                for c in range(3):
                    arrays[k][c][t.dst_at:t.dst_at + t.length].copy_(arrays[t.src][c][t.src_at:t.src_at + t.length])

    def refresh_halo(self):
        """Fill every halo copy of S from its owner (after set_spins or at the start)."""
        for k in range(self.nslabs):
            self._c[k].record(self.streams[k])
        for k in range(self.nslabs):
            self._copy(k, self.S, self._c, None)
            self._hs[k].record(self.copy_streams[k])
        self._halo_s_ready = True

    def step(self, nsteps: int = 1):
        if not self._halo_s_ready:
            self.refresh_halo()
        K = self.nslabs
        info = [s.slab_info() for s in self.slabs]
        for _ in range(int(nsteps)):
            for k in range(K):  # predictor: boundary tiles, then the core
                st, b, nt = self.streams[k], info[k]["boundary_tiles"], info[k]["num_tiles"]
                st.wait_event(self._hs[k])
                if self.early:
                    self.slabs[k].heun_pass(0, 0, b)
                    self._pb[k].record(st)
                    self.slabs[k].heun_pass(0, b, nt - b)
                else:
                    self.slabs[k].heun_pass(0, 0, nt)
                    self._pb[k].record(st)
                self._p[k].record(st)
            for k in range(K):  # S' halo: the last corrector of slab k has read its copies
                self._copy(k, self.P, self._pb, self._c if self._stepped else None)
                self._hp[k].record(self.copy_streams[k])
            for k in range(K):  # corrector: boundary tiles, then the core, then the step's end
                st, b, nt = self.streams[k], info[k]["boundary_tiles"], info[k]["num_tiles"]
                st.wait_event(self._hp[k])
                if self.early:
                    self.slabs[k].heun_pass(1, 0, b)
                    self._cb[k].record(st)
                    self.slabs[k].heun_pass(1, b, nt - b)
                else:
                    self.slabs[k].heun_pass(1, 0, nt)
                    self._cb[k].record(st)
                self.slabs[k].heun_pass(2, 0, 0)
                self._c[k].record(st)
            for k in range(K):  # S halo: the predictor of slab k has read its copies
                self._copy(k, self.S, self._cb, self._p)
                self._hs[k].record(self.copy_streams[k])
            self._stepped = True

    def sync(self):
        for k in range(self.nslabs):
            self.streams[k].synchronize()
            self.copy_streams[k].synchronize()

    # -- results ----------------------------------------------------------------------
    @property
    def step_index(self) -> int:
        return self.slabs[0].step_index

    def spins(self) -> np.ndarray:
        self.sync()
        return np.concatenate([s.spins()[:hi - lo] for s, (lo, hi) in zip(self.slabs, self.ranges)])

    def set_spins(self, S: np.ndarray):
        S = np.ascontiguousarray(S, dtype=np.float64).reshape(self.n, 3)
        self.sync()
        for s in self.slabs:
            full = s.spins()
            lo, hi = s.slab["lo"], s.slab["hi"]
            full[:hi - lo] = S[lo:hi]
            s.set_spins(full)
        self._halo_s_ready = False

    def record(self, first_step: int, count: int) -> np.ndarray:
        """(count, 1, 8) records of the whole system: the slabs' sums added in slab order."""
        self.sync()
        out = np.zeros((count, 1, 8))
        for s in self.slabs:
            out += s.record(first_step, count)
        return out


class DistributedSlab:
    """Slab ``rank`` of one system split over the ranks of a ``torch.distributed`` group.

    ``handle`` is the library handle of this rank's slab (a ``SpinSystem`` made with
    ``slab=(world, rank)`` on this rank's GPU), or any object with the same ``slab`` info,
    ``state_device``, ``heun_pass`` and ``record`` members.  Every rank builds the same
    exchange plan from the full neighbour list; a halo refresh posts one send per peer
    (that peer's runs packed, x then y then z) and one receive per peer, then unpacks."""

    def __init__(self, handle, row_ptr: np.ndarray, col: np.ndarray, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.h = handle
        n = int(np.asarray(row_ptr).size - 1)
        self.ranges = [slab_range(n, self.world, k) for k in range(self.world)]
        if (handle.slab["lo"], handle.slab["hi"]) != self.ranges[self.rank]:
            raise ValueError("the handle is not this rank's slab")
        runs = [halo_runs(row_ptr, col, lo, hi) for lo, hi in self.ranges]
        self.plan = exchange_plan(runs, self.ranges)
        self.early = sources_are_boundary(row_ptr, col, self.plan, self.ranges)
        self.send = {}  # peer -> transfers out of this slab, in plan order
        self.recv = {}  # peer -> transfers into this slab
        for t in self.plan:
            if t.src == self.rank:
                self.send.setdefault(t.dst, []).append(t)
            if t.dst == self.rank:
                self.recv.setdefault(t.src, []).append(t)
        self.S = handle.state_device(0)
        self.P = handle.state_device(1)
        if hasattr(handle, "set_stream") and self.S[0].is_cuda:
            import torch

            handle.set_stream(torch.cuda.current_stream())  # passes, packing and transfers in one order

    def _peer(self, r: int) -> int:
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def start_exchange(self, arrays):
        """Post the sends of this slab's owned runs and the receives of its halo runs."""
        import torch

        works, bufs = [], []
        for peer, ts in sorted(self.recv.items()):
            m = sum(t.length for t in ts)
            buf = torch.empty(3 * m, dtype=arrays[0].dtype, device=arrays[0].device)
            bufs.append((buf, ts, m))
            works.append(self.dist.irecv(buf, src=self._peer(peer), group=self.group))
        for peer, ts in sorted(self.send.items()):
            pk = torch.cat([arrays[c][t.src_at:t.src_at + t.length] for c in range(3) for t in ts])
            works.append(self.dist.isend(pk, dst=self._peer(peer), group=self.group))
            bufs.append((pk, None, 0))  # the send buffer lives until the transfer ends
        return works, bufs, arrays

    def finish_exchange(self, pending):
        works, bufs, arrays = pending
        for w in works:
            w.wait()
        for buf, ts, m in bufs:
            if ts is None:
                continue
            for c in range(3):
                at = c * m
                for t in ts:
                    arrays[c][t.dst_at:t.dst_at + t.length].copy_(buf[at:at + t.length])
                    at += t.length

    def refresh_halo(self):
        self.finish_exchange(self.start_exchange(self.S))

    def step(self, nsteps: int = 1):
        info = self.h.slab_info() if hasattr(self.h, "slab_info") else self.h.slab
        b, nt = info["boundary_tiles"], info["num_tiles"]
        if not self.early:
            b = nt
        for _ in range(int(nsteps)):
            self.h.heun_pass(0, 0, b)
            pending = self.start_exchange(self.P)
            self.h.heun_pass(0, b, nt - b)
            self.finish_exchange(pending)
            self.h.heun_pass(1, 0, b)
            pending = self.start_exchange(self.S)
            self.h.heun_pass(1, b, nt - b)
            self.h.heun_pass(2, 0, 0)
            self.finish_exchange(pending)

    def record(self, first_step: int, count: int):
        """(count, 1, 8) records of the whole system: this slab's sums all-reduced over the
        group (every rank gets the same array)."""
        import torch

        local = torch.as_tensor(np.ascontiguousarray(self.h.record(first_step, count)), dtype=torch.float64)
        dev = self.S[0].device
        t = local.to(dev)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

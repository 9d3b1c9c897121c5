"""User-facing Python front end of libspinsys (argument marshalling only).

``SpinSystem`` owns one C handle (one system, or a batch of independent systems) and
forwards every call to the C ABI of ``include/spinsys.h``.  Arrays come from
``paper_1310_6143_gb300.lattice`` (or any source of the same shapes).  PyTorch is only
used, when asked, for the CUDA stream handle and zero-copy device views of the spins.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _binding as B
from .lattice import SpinLattice

_PREC = {"fp64": B.SS_FP64, "fp32": B.SS_FP32_MIXED, "fp32_mixed": B.SS_FP32_MIXED}
_EXEC = {"auto": B.SS_EXEC_AUTO, "kernels": B.SS_EXEC_KERNELS, "graph": B.SS_EXEC_GRAPH,
         "persistent": B.SS_EXEC_PERSISTENT, "system_blocks": B.SS_EXEC_SYSTEM_BLOCKS, "cluster": B.SS_EXEC_CLUSTER}


def _per_system(v, count, name):
    if isinstance(v, (list, tuple, np.ndarray)) and np.ndim(v) >= 1 and not (
            name == "H" and np.ndim(v) == 1 and len(v) == 3 and count != 3):
        if name == "H" and np.ndim(v) == 1:
            return [tuple(v)] * count
        if len(v) != count:
            raise ValueError(f"{name}: need one value per system ({count})")
        return list(v)
    return [v] * count


class _DeviceArray:
    """Minimal __cuda_array_interface__ carrier for zero-copy torch views."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


class SpinSystem:
    """One handle of the GB300 Heun-LLG library.

    ``lattices`` is a SpinLattice or a sequence of them (a batch of independent systems).
    ``alpha``, ``dt``, ``T``, ``H``, ``seed``, ``sys_id`` and ``S0`` may be given per
    system as sequences.  ``precision`` is "fp64" or "fp32" (FP32 storage and field/LLG
    arithmetic with FP64 thermal transform and FP64 reductions).
    ``slab=(nslabs, index)`` makes the handle of one slab of a single lattice (the owned
    global range plus halo copies, advanced by ``heun_pass``; see ``paper_1310_6143_gb300.slab``).
    """

    def __init__(self, lattices: SpinLattice | Sequence[SpinLattice], *, alpha=0.1, dt=1e-16, T=0.0,
                 H=(0.0, 0.0, 0.0), seed=1, sys_id=None, precision="fp64", S0=None, init_random=False,
                 gamma=0.0, check_symmetry=False, stream=None, slab=None):
        self._lib = B.load()
        self._h = ctypes.c_void_p()
        lats = [lattices] if isinstance(lattices, SpinLattice) else list(lattices)
        count = len(lats)
        if count < 1:
            raise ValueError("need at least one lattice")
        alphas = _per_system(alpha, count, "alpha")
        dts = _per_system(dt, count, "dt")
        Ts = _per_system(T, count, "T")
        Hs = _per_system(H, count, "H")
        seeds = _per_system(seed, count, "seed")
        ids = list(range(count)) if sys_id is None else _per_system(sys_id, count, "sys_id")
        S0s = [None] * count if S0 is None else (list(S0) if count > 1 else [S0])
        if len(S0s) != count:
            raise ValueError(f"S0: need one initial state per system ({count})")
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {sorted(_PREC)}")
        keep = []
        params = (B.SSParams * count)()
        for s, lat in enumerate(lats):
            arrs = {
                "row_ptr": np.ascontiguousarray(lat.row_ptr, dtype=np.int64),
                "col": np.ascontiguousarray(lat.col, dtype=np.int32),
                "J": np.ascontiguousarray(lat.J, dtype=np.float64),
                "mu_s": np.ascontiguousarray(lat.mu_s, dtype=np.float64),
                "k_u": np.ascontiguousarray(lat.k_u, dtype=np.float64),
                "easy_axis": np.ascontiguousarray(lat.easy_axis, dtype=np.float64),
                "K_neel": None if lat.K_neel is None else np.ascontiguousarray(lat.K_neel, dtype=np.float64),
                "pos": None if lat.pos is None else np.ascontiguousarray(lat.pos, dtype=np.float64),
                "S0": None if S0s[s] is None else np.ascontiguousarray(S0s[s], dtype=np.float64),
                "J_tensor": None if lat.J_tensor is None else np.ascontiguousarray(lat.J_tensor, dtype=np.float64),
                "k_c": None if lat.k_c is None else np.ascontiguousarray(lat.k_c, dtype=np.float64),
            }
            keep.append(arrs)
            p = params[s]
            p.n = lat.n
            for k, a in arrs.items():
                setattr(p, k, None if a is None else a.ctypes.data)
            p.alpha = float(alphas[s])
            p.dt = float(dts[s])
            p.gamma = float(gamma)
            for c in range(3):
                p.H_app[c] = float(Hs[s][c])
            p.T = float(Ts[s])
            p.seed = int(seeds[s]) & 0xFFFFFFFFFFFFFFFF
            p.sys_id = int(ids[s]) & 0xFFFFFFFF
            p.precision = _PREC[precision]
            p.flags = (B.SS_FLAG_CHECK_SYMMETRY if check_symmetry else 0) | (B.SS_FLAG_INIT_RANDOM if init_random else 0)
        if slab is not None:
            if count != 1:
                raise ValueError("a slab handle decomposes one lattice")
            st = self._lib.spin_slab_create(ctypes.byref(params[0]), int(slab[0]), int(slab[1]), ctypes.byref(self._h))
        elif count == 1:
            st = self._lib.spin_system_create(ctypes.byref(params[0]), ctypes.byref(self._h))
        else:
            st = self._lib.spin_batch_create(params, count, ctypes.byref(self._h))
        B.check(st, None)
        self.n = int(sum(l.n for l in lats))
        self.slab = None
        if slab is not None:
            si = self.slab_info()
            self.n = int(si["hi"] - si["lo"] + si["n_halo"])  # owned spins, then the halo copies
        self.num_systems = count
        self.sizes = [l.n for l in lats]
        self.offsets = list(np.cumsum([0] + self.sizes[:-1]))
        self.precision = precision
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime ---------------------------------------------------------------------
    def close(self):
        if self._h:
            self._lib.spin_system_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        B.check(st, self._h)

    # -- configuration ----------------------------------------------------------------
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (own stream)."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.spin_system_set_stream(self._h, ctypes.c_void_p(raw) if raw else None))
        self._stream = stream  # the handle launches on it: keep the owner alive as long as the handle

    def set_field(self, H, sys: int = -1):
        arr = np.ascontiguousarray(H, dtype=np.float64).reshape(3)
        self._check(self._lib.set_field(self._h, int(sys), B.ptr(arr)))

    def set_temperature(self, T):
        if np.ndim(T) == 0:
            self._check(self._lib.set_temperature(self._h, float(T)))
        else:
            arr = np.ascontiguousarray(T, dtype=np.float64)
            self._check(self._lib.set_temperature_batch(self._h, B.ptr(arr), int(arr.size)))

    def set_temperature_schedule(self, T_per_step, step0: int = 0):
        arr = np.ascontiguousarray(T_per_step, dtype=np.float64)
        self._check(self._lib.set_temperature_schedule(self._h, B.ptr(arr), int(arr.size), int(step0)))

    def set_exec(self, mode: str):
        self._check(self._lib.spin_system_set_exec(self._h, _EXEC[mode]))

    def set_launch(self, block: int, tile: int):
        self._check(self._lib.spin_system_set_launch(self._h, int(block), int(tile)))

    def set_exchange_rows(self, mode: str):
        """'auto', 'thread' (a thread per exchange row) or 'warp' (a warp per row)."""
        self._check(self._lib.spin_system_set_exchange_rows(self._h, {"auto": 0, "thread": 1, "warp": 2}[mode]))

    def set_gaussian_pass(self, mode):
        """FP32-mixed: 0/False the Heun passes draw the Gaussians (the default), 1/True a
        separate pass writes each step's Gaussians first, 2 that pass runs concurrently with
        the previous step."""
        self._check(self._lib.spin_system_set_gaussian_pass(self._h, int(mode)))

    def time_passes(self, nsteps: int) -> dict:
        """Real steps with CUDA events around every launch: mean Gaussian-pass, predictor and
        corrector launch times and mean step time, in ms."""
        out = np.zeros(4)
        self._check(self._lib.spin_system_time_passes(self._h, int(nsteps), B.ptr(out)))
        return {"gauss_ms": out[0], "predictor_ms": out[1], "corrector_ms": out[2], "step_ms": out[3]}

    def set_row_patterns(self, on: bool):
        """Read the row forms (True, the default when they were built) or the CSR."""
        self._check(self._lib.spin_system_set_row_patterns(self._h, 1 if on else 0))

    def set_draw_ahead(self, eighths: int):
        self._check(self._lib.spin_system_set_draw_ahead(self._h, int(eighths)))

    def autotune(self, trial_steps: int = 20) -> dict:
        info = B.SSInfo()
        self._check(self._lib.spin_system_autotune(self._h, int(trial_steps), ctypes.byref(info)))
        return info.as_dict()

    def info(self) -> dict:
        info = B.SSInfo()
        self._check(self._lib.spin_system_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def time_kernels(self, nsteps: int) -> dict:
        """Real steps with CUDA events around every launch: mean predictor / corrector
        launch time and mean step time, in ms."""
        out = np.zeros(3)
        self._check(self._lib.spin_system_time_kernels(self._h, int(nsteps), B.ptr(out)))
        return {"predictor_ms": out[0], "corrector_ms": out[1], "step_ms": out[2]}

    def time_rows(self, launches: int = 10) -> float:
        """Mean duration (ms) of one warp-per-row exchange pass over the current spins."""
        out = np.zeros(1)
        self._check(self._lib.spin_system_time_rows(self._h, int(launches), B.ptr(out)))
        return float(out[0])

    def set_barrier_test(self, extra: int, timeout_ns: int):
        self._check(self._lib.spin_system_set_barrier_test(self._h, int(extra), int(timeout_ns)))

    # -- stepping and state -----------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._lib.llg_heun_step(self._h, int(n)))

    def set_demag(self, cell_size: float, atom_volume: float, every: int = 1):
        """Macrocell demagnetising field: cubic cells of edge cell_size (m), volume per atom
        atom_volume (m^3), recomputed every `every` steps; cell_size <= 0 switches it off.
        Needs the lattices' positions."""
        self._check(self._lib.set_demag(self._h, float(cell_size), float(atom_volume), int(every)))

    def demag_field(self) -> np.ndarray:
        """The demagnetising field in force, per atom, (n, 3) tesla."""
        out = np.zeros((self.n, 3))
        self._check(self._lib.get_demag_field(self._h, B.ptr(out)))
        return out

    def midpoint_step(self, n: int = 1, iterations: int = 4):
        """n steps of the midpoint rule (fixed-point iterations per step), instead of Heun."""
        self._check(self._lib.llg_midpoint_step(self._h, int(n), int(iterations)))

    def semi_implicit_step(self, n: int = 1):
        """n steps of the semi-implicit predictor-corrector scheme (Mentink et al.), instead of Heun."""
        self._check(self._lib.llg_semi_implicit_step(self._h, int(n)))

    def mc_step(self, n: int = 1):
        """n Hinzke-Nowak Monte Carlo steps (one trial move per spin each)."""
        self._check(self._lib.mc_step(self._h, int(n)))

    def mc_stats(self, sys: int = 0):
        """(accepted, attempted) Monte Carlo trial moves of system `sys` so far."""
        out = (ctypes.c_int64 * 2)()
        self._check(self._lib.get_mc_stats(self._h, int(sys), out))
        return int(out[0]), int(out[1])

    def sync(self):
        self._check(self._lib.spin_system_sync(self._h))

    @property
    def step_index(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.get_step(self._h, ctypes.byref(v)))
        return int(v.value)

    @step_index.setter
    def step_index(self, step: int):
        self._check(self._lib.set_step(self._h, int(step)))

    def spins(self, out: np.ndarray | None = None) -> np.ndarray:
        out = np.empty((self.n, 3)) if out is None else out
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 3 * self.n
        self._check(self._lib.get_spins(self._h, B.ptr(out)))
        return out

    def set_spins(self, S: np.ndarray):
        arr = np.ascontiguousarray(S, dtype=np.float64).reshape(self.n, 3)
        self._check(self._lib.set_spins(self._h, B.ptr(arr)))

    def spins_device(self):
        """Zero-copy torch views (x, y, z) of the device spins, valid until the next step."""
        import torch

        px, py, pz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._check(self._lib.get_spins_device(self._h, ctypes.byref(px), ctypes.byref(py), ctypes.byref(pz)))
        ts = "<f4" if self.precision != "fp64" else "<f8"
        return tuple(torch.as_tensor(_DeviceArray(p.value, self.n, ts), device="cuda") for p in (px, py, pz))

    def state_device(self, which: int = 0):
        """Zero-copy torch views (x, y, z) of the state S (which=0) or the predictor spins S'
        (which=1); the buffers live as long as the handle."""
        import torch

        px, py, pz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._check(self._lib.get_state_device(self._h, int(which), ctypes.byref(px), ctypes.byref(py),
                                               ctypes.byref(pz)))
        ts = "<f4" if self.precision != "fp64" else "<f8"
        return tuple(torch.as_tensor(_DeviceArray(p.value, self.n, ts), device="cuda") for p in (px, py, pz))

    def slab_info(self) -> dict:
        """The slab's ranges and tile split (refreshed: a new launch shape re-tiles)."""
        si = B.SSSlabInfo()
        self._check(self._lib.spin_slab_info(self._h, ctypes.byref(si)))
        self.slab = si.as_dict()
        return self.slab

    def halo_runs(self) -> np.ndarray:
        """(num_runs, 3) int64: first global index, length, first local index of each halo run."""
        nr = int(self.slab["num_runs"]) if self.slab else 0
        out = np.zeros((max(nr, 1), 3), dtype=np.int64)
        self._check(self._lib.spin_slab_halo_runs(self._h, B.ptr(out), nr))
        return out[:nr]

    def heun_pass(self, which: int, tile0: int, ntiles: int):
        """Enqueue pass ``which`` (0 predictor, 1 corrector, 2 end of step) over tiles
        [tile0, tile0 + ntiles) on the handle's stream."""
        self._check(self._lib.spin_system_heun_pass(self._h, int(which), int(tile0), int(ntiles)))

    def magnetisation(self, sys: int = 0) -> np.ndarray:
        out = np.zeros(4)
        self._check(self._lib.get_magnetisation(self._h, int(sys), B.ptr(out)))
        return out

    def energy(self, sys: int = 0) -> np.ndarray:
        out = np.zeros(4)
        self._check(self._lib.get_energy(self._h, int(sys), B.ptr(out)))
        return out

    def record(self, first_step: int, count: int) -> np.ndarray:
        """(count, num_systems, 8): sum mu S (3), sum mu, E_exc, E_ani, E_app, E_total."""
        out = np.zeros((count, self.num_systems, 8))
        self._check(self._lib.get_record(self._h, int(first_step), int(count), B.ptr(out)))
        return out


def debug_philox(ctr0, key, count: int) -> np.ndarray:
    lib = B.load()
    c = np.ascontiguousarray(ctr0, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((count, 4), dtype=np.uint32)
    B.check(lib.ss_debug_philox(B.ptr(c), B.ptr(k), int(count), B.ptr(out)))
    return out


def debug_gaussians(seed: int, sys_id: int, step: int, n: int, mode: int = 0) -> np.ndarray:
    lib = B.load()
    out = np.zeros((n, 3))
    B.check(lib.ss_debug_gaussians(int(seed) & 0xFFFFFFFFFFFFFFFF, int(sys_id), int(step), int(n), int(mode),
                                   B.ptr(out)))
    return out


def debug_fp64_rate(mode: int = 1) -> float:
    """Measured FP64 instructions per second of the current device (see spinsys.h)."""
    lib = B.load()
    out = ctypes.c_double()
    B.check(lib.ss_debug_fp64_rate(int(mode), ctypes.byref(out)))
    return out.value

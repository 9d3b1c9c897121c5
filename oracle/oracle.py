"""ctypes front end of ``spinsys_oracle.c`` (test infrastructure only).

The C file is compiled with ``gcc -O3 -ffp-contract=off`` so that every product and sum
is rounded exactly as written; see the header of ``spinsys_oracle.c`` for the equations
of arXiv:1310.6143 it follows and the readings it takes where the paper is silent.
Arrays are array-of-structures: spins ``(n, 3)``, easy axes ``(n, 3)``, Neel tensors
``(n, 6)`` in the order xx, yy, zz, xy, xz, yz.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spinsys_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


# -O3 with no FMA contraction and no value-changing optimisation: every product and sum is
# rounded as written, so the results are those of the -O2 build bit for bit (checked by a CPU
# test).  No -march=native: the oracle must give the same results on x86 and Arm hosts.
FLAGS = ["-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stamp = _LIB + ".flags"
    flags_now = " ".join(FLAGS)
    stale = not os.path.exists(stamp) or open(stamp).read() != flags_now
    if force or stale or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", *FLAGS, "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(flags_now)
    return _LIB


class _CSys(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("J", ctypes.c_void_p),
        ("mu_s", ctypes.c_void_p),
        ("k_u", ctypes.c_void_p),
        ("easy_axis", ctypes.c_void_p),
        ("K_neel", ctypes.c_void_p),
        ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("H_app", ctypes.c_double * 3),
        ("seed", ctypes.c_uint64),
        ("sys", ctypes.c_uint32),
        ("ids", ctypes.c_void_p),
        ("pos", ctypes.c_void_p),
        ("demag_cell", ctypes.c_double),
        ("demag_vatom", ctypes.c_double),
        ("demag_every", ctypes.c_int64),
        ("Jt", ctypes.c_void_p),
        ("k_c", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # SPINSYS_ORACLE_LIB names a prebuilt oracle library to use instead (the mutation
            # test loads deliberately broken copies this way, in child processes)
            lib = ctypes.CDLL(os.environ.get("SPINSYS_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_thermal_gaussians.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                                  ctypes.c_uint32, P]
            lib.orc_init_sphere.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, P]
            lib.orc_fields.argtypes = [ctypes.POINTER(_CSys), P, P]
            lib.orc_moment_energy.argtypes = [ctypes.POINTER(_CSys), P, P]
            lib.orc_heun_run.argtypes = [ctypes.POINTER(_CSys), P, ctypes.c_int64, ctypes.c_int64, P, P]
            lib.orc_heun_run.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            lib.orc_philox_bulk.argtypes = [P, P, ctypes.c_int64, P]
            lib.orc_gaussians_bulk.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_int64, P]
            lib.orc_colour_greedy.argtypes = [ctypes.POINTER(_CSys), P]
            lib.orc_colour_greedy.restype = ctypes.c_int
            lib.orc_mc_sigma_g.argtypes = [ctypes.c_double]
            lib.orc_mc_sigma_g.restype = ctypes.c_double
            lib.orc_mc_run.argtypes = [ctypes.POINTER(_CSys), P, ctypes.c_int64, ctypes.c_int64, P, P,
                                       ctypes.c_int32, P, P]
            lib.orc_mc_run.restype = ctypes.c_int
            lib.orc_midpoint_run.argtypes = [ctypes.POINTER(_CSys), P, ctypes.c_int64, ctypes.c_int64, P,
                                             ctypes.c_int, P]
            lib.orc_midpoint_run.restype = ctypes.c_int
            lib.orc_sib_run.argtypes = [ctypes.POINTER(_CSys), P, ctypes.c_int64, ctypes.c_int64, P, P]
            lib.orc_sib_run.restype = ctypes.c_int
            lib.orc_macrocells.argtypes = [ctypes.POINTER(_CSys), P]
            lib.orc_macrocells.restype = ctypes.c_int64
            lib.orc_demag_fields.argtypes = [ctypes.POINTER(_CSys), P, P, P]
            lib.orc_demag_fields.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class OracleSystem:
    """One spin system in SI units (J/T, J, T, s), arrays as numpy float64/int."""

    row_ptr: np.ndarray
    col: np.ndarray
    J: np.ndarray
    mu_s: np.ndarray
    k_u: np.ndarray
    easy_axis: np.ndarray
    K_neel: np.ndarray | None = None
    alpha: float = 0.1
    dt: float = 1e-16
    gamma: float = 1.76e11
    H_app: tuple = (0.0, 0.0, 0.0)
    seed: int = 1
    sys_id: int = 0
    ids: np.ndarray | None = None
    pos: np.ndarray | None = None       # (n, 3) atomic positions, m (demagnetising field)
    demag_cell: float = 0.0             # macrocell edge, m; 0: no demagnetising field
    demag_vatom: float = 0.0            # volume per atom, m^3
    demag_every: int = 1                # steps between demagnetising-field updates
    J_tensor: np.ndarray | None = None  # (nnz, 3, 3) exchange tensors, or None (scalar J)
    k_c: np.ndarray | float | None = None  # cubic anisotropy, J/atom
    _keep: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        self.row_ptr = np.ascontiguousarray(self.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(self.col, dtype=np.int32)
        self.J = np.ascontiguousarray(self.J, dtype=np.float64)
        n = self.row_ptr.size - 1
        self.mu_s = np.ascontiguousarray(np.broadcast_to(np.asarray(self.mu_s, dtype=np.float64), (n,)))
        self.k_u = np.ascontiguousarray(np.broadcast_to(np.asarray(self.k_u, dtype=np.float64), (n,)))
        self.easy_axis = np.ascontiguousarray(
            np.broadcast_to(np.asarray(self.easy_axis, dtype=np.float64), (n, 3)))
        if self.K_neel is not None:
            self.K_neel = np.ascontiguousarray(self.K_neel, dtype=np.float64).reshape(n, 6)
        if self.ids is not None:
            self.ids = np.ascontiguousarray(self.ids, dtype=np.uint32).reshape(n)
        if self.pos is not None:
            self.pos = np.ascontiguousarray(self.pos, dtype=np.float64).reshape(n, 3)
        if self.J_tensor is not None:
            self.J_tensor = np.ascontiguousarray(self.J_tensor, dtype=np.float64).reshape(-1, 3, 3)
        if self.k_c is not None:
            self.k_c = np.ascontiguousarray(np.broadcast_to(np.asarray(self.k_c, dtype=np.float64), (n,)))

    @property
    def n(self) -> int:
        return self.row_ptr.size - 1

    def _c(self) -> _CSys:
        c = _CSys()
        c.n = self.n
        c.row_ptr = _ptr(self.row_ptr)
        c.col = _ptr(self.col)
        c.J = _ptr(self.J)
        c.mu_s = _ptr(self.mu_s)
        c.k_u = _ptr(self.k_u)
        c.easy_axis = _ptr(self.easy_axis)
        c.K_neel = _ptr(self.K_neel)
        c.alpha = float(self.alpha)
        c.dt = float(self.dt)
        c.gamma = float(self.gamma)
        for k in range(3):
            c.H_app[k] = float(self.H_app[k])
        c.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        c.sys = int(self.sys_id) & 0xFFFFFFFF
        c.ids = _ptr(self.ids)
        c.pos = _ptr(self.pos)
        c.demag_cell = float(self.demag_cell)
        c.demag_vatom = float(self.demag_vatom)
        c.demag_every = int(self.demag_every)
        c.Jt = _ptr(self.J_tensor)
        c.k_c = _ptr(self.k_c)
        return c


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under a 64-bit key -> 4 uint32 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_bulk(ctr0, key, count: int) -> np.ndarray:
    """Philox4x32-10 of counters (c0+k, c1, c2, c3), k < count -> (count, 4) uint32."""
    c = np.ascontiguousarray(ctr0, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros((count, 4), dtype=np.uint32)
    _load().orc_philox_bulk(_ptr(c), _ptr(k), int(count), _ptr(out))
    return out


def gaussians_bulk(seed: int, sys_id: int, step: int, n: int) -> np.ndarray:
    """Thermal Gaussian triples of spins 0..n-1 at one step -> (n, 3)."""
    g = np.zeros((n, 3))
    _load().orc_gaussians_bulk(int(seed) & 0xFFFFFFFFFFFFFFFF, int(sys_id), int(step), int(n), _ptr(g))
    return g


def thermal_gaussians(seed: int, sys_id: int, spin: int, step: int) -> np.ndarray:
    g = np.zeros(3)
    _load().orc_thermal_gaussians(int(seed) & 0xFFFFFFFFFFFFFFFF, int(sys_id), int(spin), int(step), _ptr(g))
    return g


def init_sphere(seed: int, sys_id: int, n: int) -> np.ndarray:
    S = np.zeros((n, 3))
    _load().orc_init_sphere(int(seed) & 0xFFFFFFFFFFFFFFFF, int(sys_id), int(n), _ptr(S))
    return S


def fields(system: OracleSystem, S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(system.n, 3)
    H = np.zeros_like(S)
    c = system._c()
    _load().orc_fields(ctypes.byref(c), _ptr(S), _ptr(H))
    return H


def moment_energy(system: OracleSystem, S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(system.n, 3)
    out = np.zeros(8)
    c = system._c()
    _load().orc_moment_energy(ctypes.byref(c), _ptr(S), _ptr(out))
    return out


def heun_run(system: OracleSystem, S: np.ndarray, nsteps: int, T, step0: int = 0,
             record: bool = False):
    """Advance ``nsteps`` Heun steps; returns (S_new, rec or None).

    ``T`` is a scalar temperature (K) or an array of ``nsteps`` temperatures.
    ``rec`` has shape (nsteps, 8): moment and energy of the state at the start of each step.
    """
    S = np.array(S, dtype=np.float64, copy=True).reshape(system.n, 3)
    Tarr = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (nsteps,)))
    rec = np.zeros((nsteps, 8)) if record else None
    c = system._c()
    rc = _load().orc_heun_run(ctypes.byref(c), _ptr(S), int(step0), int(nsteps), _ptr(Tarr), _ptr(rec))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return S, rec


def midpoint_run(system: OracleSystem, S: np.ndarray, nsteps: int, T, iters: int = 4, step0: int = 0,
                 record: bool = False):
    """Advance ``nsteps`` midpoint-rule steps with ``iters`` fixed-point iterations each;
    returns (S_new, rec or None) as heun_run."""
    S = np.array(S, dtype=np.float64, copy=True).reshape(system.n, 3)
    Tarr = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (nsteps,)))
    rec = np.zeros((nsteps, 8)) if record else None
    c = system._c()
    rc = _load().orc_midpoint_run(ctypes.byref(c), _ptr(S), int(step0), int(nsteps), _ptr(Tarr), int(iters),
                                  _ptr(rec))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return S, rec


def sib_run(system: OracleSystem, S: np.ndarray, nsteps: int, T, step0: int = 0, record: bool = False):
    """Advance ``nsteps`` semi-implicit predictor-corrector steps (Mentink et al.'s scheme B);
    returns (S_new, rec or None) as heun_run."""
    S = np.array(S, dtype=np.float64, copy=True).reshape(system.n, 3)
    Tarr = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (nsteps,)))
    rec = np.zeros((nsteps, 8)) if record else None
    c = system._c()
    rc = _load().orc_sib_run(ctypes.byref(c), _ptr(S), int(step0), int(nsteps), _ptr(Tarr), _ptr(rec))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return S, rec


def colour_greedy(system: OracleSystem):
    """Greedy colouring of the neighbour graph in site order -> (colour[n] int32, ncolours)."""
    colour = np.zeros(system.n, dtype=np.int32)
    c = system._c()
    nc = _load().orc_colour_greedy(ctypes.byref(c), _ptr(colour))
    if nc < 0:
        raise MemoryError("oracle: allocation failed")
    return colour, int(nc)


def mc_sigma_g(T: float) -> float:
    """Width of the Gaussian trial cone at temperature T (Eq. MCgaussianSigma)."""
    return float(_load().orc_mc_sigma_g(float(T)))


def mc_run(system: OracleSystem, S: np.ndarray, nsteps: int, T, step0: int = 0, record: bool = False):
    """Advance ``nsteps`` Hinzke-Nowak Monte Carlo steps; returns (S_new, rec or None, accepted).

    ``T`` is a scalar temperature (K) or an array of ``nsteps`` temperatures; ``accepted``
    holds the accepted trial moves of each step (one trial per spin per step).
    """
    S = np.array(S, dtype=np.float64, copy=True).reshape(system.n, 3)
    Tarr = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (nsteps,)))
    colour, nc = colour_greedy(system)
    rec = np.zeros((nsteps, 8)) if record else None
    acc = np.zeros(nsteps, dtype=np.int64)
    c = system._c()
    rc = _load().orc_mc_run(ctypes.byref(c), _ptr(S), int(step0), int(nsteps), _ptr(Tarr), _ptr(colour), nc,
                            _ptr(rec), _ptr(acc))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return S, rec, acc


def macrocells(system: OracleSystem):
    """Macrocell of every atom (needs ``pos`` and ``demag_cell``) -> (cell[n] int64, ncell)."""
    cell = np.zeros(system.n, dtype=np.int64)
    c = system._c()
    nc = _load().orc_macrocells(ctypes.byref(c), _ptr(cell))
    if nc < 0:
        raise MemoryError("oracle: allocation failed")
    return cell, int(nc)


def demag_fields(system: OracleSystem, S: np.ndarray):
    """Macrocell demagnetising field of the state S -> (per atom (n, 3), per macrocell (ncell, 3)), T."""
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(system.n, 3)
    _, nc = macrocells(system)
    Hd = np.zeros((system.n, 3))
    Hmc = np.zeros((max(nc, 1), 3))
    c = system._c()
    if _load().orc_demag_fields(ctypes.byref(c), _ptr(S), _ptr(Hd), _ptr(Hmc)) < 0:
        raise MemoryError("oracle: allocation failed")
    return Hd, Hmc[:nc]

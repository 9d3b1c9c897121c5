"""llg_heun_step_noalloc: the allocation-free FP64 step, checked against llg_heun_step.

Callers that cannot allocate device memory (code inside an arena that owns all device
memory, loops that must not allocate after start-up) pass their own device arrays and
let the library keep its working buffers in a static device array.  This test plays
such a caller: it holds the system's arrays in device memory (allocated here, by the
test, with torch), calls the new entry point twice in a row through the C ABI, and
compares spins and per-step records with a handle created by spin_system_create and
advanced by llg_heun_step, within the FP64 parity tolerance of the other tests (1e-12).
Around the second call the device's free memory does not change (an allocation of the
working buffers, 9.5 MB, would show).  It also checks that a system larger than
SS_NOALLOC_MAX_SPINS, and steps past the 32-bit counter, are refused.
"""
import ctypes

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu

TOL = 1e-12
MAX_SPINS = 131072


class NoAllocStep(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("J", ctypes.c_void_p),
        ("mu_s", ctypes.c_void_p),
        ("k_u", ctypes.c_void_p),
        ("easy_axis", ctypes.c_void_p),
        ("sx", ctypes.c_void_p),
        ("sy", ctypes.c_void_p),
        ("sz", ctypes.c_void_p),
        ("record", ctypes.c_void_p),
        ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("H_app", ctypes.c_double * 3),
        ("T", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("sys_id", ctypes.c_uint32),
        ("step0", ctypes.c_int64),
    ]


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6143_gb300 import _binding as B

    lib = B.load()
    lib.llg_heun_step_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.llg_heun_step_noalloc.restype = ctypes.c_int
    return lib


def _system():
    lat = L.simple_cubic(11, 9, 7, J=6.0e-21, k_u=2.0e-23)  # 693 spins: a ragged last tile
    rng = np.random.default_rng(3)
    ax = rng.normal(size=(lat.n, 3))
    lat.easy_axis = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    lat.mu_s = rng.uniform(1.0, 2.0, lat.n) * L.MU_B
    return lat


def test_noalloc_matches_handle_two_calls(lib):
    import torch

    from paper_1310_6143_gb300.system import SpinSystem

    lat = _system()
    n = lat.n
    S0 = L.random_state(n, 7)
    kw = dict(alpha=0.1, dt=1e-16, T=400.0, H=(0.3, 0.0, 1.0), seed=11, sys_id=2)
    k1, k2 = 40, 25
    with SpinSystem(lat, precision="fp64", S0=S0, **kw) as s:
        s.step(k1)
        ref1 = s.spins()
        s.step(k2)
        ref2 = s.spins()
        rec_ref = s.record(0, k1 + k2)[:, 0, :]
        axes = lat.easy_axis / np.linalg.norm(lat.easy_axis, axis=1, keepdims=True)

    dev = torch.device("cuda")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    row_ptr = t(lat.row_ptr, torch.int32)
    col = t(lat.col, torch.int32)
    J = t(lat.J, torch.float64)
    mu = t(lat.mu_s, torch.float64)
    ku = t(lat.k_u, torch.float64)
    ea = t(axes.reshape(-1), torch.float64)
    S = [t(S0[:, c], torch.float64) for c in range(3)]
    rec = torch.zeros((k1 + k2, 8), dtype=torch.float64, device=dev)

    p = NoAllocStep()
    p.n = n
    p.row_ptr, p.col, p.J = row_ptr.data_ptr(), col.data_ptr(), J.data_ptr()
    p.mu_s, p.k_u, p.easy_axis = mu.data_ptr(), ku.data_ptr(), ea.data_ptr()
    p.sx, p.sy, p.sz = (x.data_ptr() for x in S)
    p.alpha, p.dt, p.gamma, p.T = kw["alpha"], kw["dt"], 0.0, kw["T"]
    for c in range(3):
        p.H_app[c] = kw["H"][c]
    p.seed, p.sys_id = kw["seed"], kw["sys_id"]
    stream = torch.cuda.current_stream().cuda_stream

    # first call: steps 0 .. k1-1
    p.step0 = 0
    p.record = rec.data_ptr()
    assert lib.llg_heun_step_noalloc(ctypes.byref(p), k1, ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    got1 = torch.stack(S, 1).cpu().numpy()
    assert np.abs(got1 - ref1).max() <= TOL
    # second call continues from the first call's output: steps k1 .. k1+k2-1
    p.step0 = k1
    p.record = rec.data_ptr() + k1 * 8 * 8
    free_before = torch.cuda.mem_get_info()[0]
    assert lib.llg_heun_step_noalloc(ctypes.byref(p), k2, ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before  # nothing allocated on the device
    got2 = torch.stack(S, 1).cpu().numpy()
    assert np.abs(got2 - ref2).max() <= TOL
    r = rec.cpu().numpy()
    scale_m = rec_ref[:, 3].max()
    scale_e = np.abs(rec_ref[:, 4:7]).max()
    assert np.abs(r[:, :4] - rec_ref[:, :4]).max() <= TOL * scale_m
    assert np.abs(r[:, 4:] - rec_ref[:, 4:]).max() <= TOL * scale_e


def test_noalloc_rejects_oversized_system(lib):
    from paper_1310_6143_gb300 import _binding as B

    p = NoAllocStep()
    p.n = MAX_SPINS + 1
    p.dt = 1e-16
    st = lib.llg_heun_step_noalloc(ctypes.byref(p), 1, None)
    assert st == 1  # SS_ERR_INVALID_ARG
    assert "SS_NOALLOC_MAX_SPINS" in B.load().ss_last_error(None).decode()


def test_noalloc_rejects_steps_past_the_counter(lib):
    p = NoAllocStep()
    p.n = 8
    p.dt = 1e-16
    p.row_ptr = p.col = p.J = p.mu_s = p.k_u = p.easy_axis = p.sx = p.sy = p.sz = 1  # never dereferenced
    p.step0 = 2**32 - 3
    assert lib.llg_heun_step_noalloc(ctypes.byref(p), 3, None) == 1  # SS_ERR_INVALID_ARG: step 2^32 - 1

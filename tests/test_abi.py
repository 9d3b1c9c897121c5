"""C ABI checks that need no GPU: the library builds for sm_103a, exports every entry
point include/spinsys.h declares, and rejects invalid input on the host before any CUDA
call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6143_gb300 import _binding as B
    from paper_1310_6143_gb300 import build

    build.build()
    return B.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "spinsys.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"^\s*(?:ss_status|const char \*|int64_t)\s*(\w+)\s*\(", txt, flags=re.M))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("spin_system_create", "set_field", "set_temperature", "llg_heun_step", "get_spins",
                     "get_magnetisation", "get_energy", "spin_batch_create"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1310_6143_gb300 import _binding as B

    names = _declared()
    assert names == set(B.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_host_validation_without_gpu(lib):
    from paper_1310_6143_gb300 import _binding as B
    from paper_1310_6143_gb300 import lattice as L

    lat = L.simple_cubic(3, 3, 3)

    def create(**over):
        arrs = dict(row_ptr=lat.row_ptr.copy(), col=lat.col.copy(), J=lat.J.copy(), mu_s=lat.mu_s.copy(),
                    k_u=lat.k_u.copy(), easy_axis=lat.easy_axis.copy())
        scal = dict(n=lat.n, alpha=0.1, dt=1e-16, T=0.0)
        for k, v in over.items():
            (arrs if k in arrs else scal)[k] = v
        p = B.SSParams()
        for k, v in arrs.items():
            setattr(p, k, v.ctypes.data)
        for k, v in scal.items():
            setattr(p, k, v)
        h = ctypes.c_void_p()
        st = lib.spin_system_create(ctypes.byref(p), ctypes.byref(h))
        msg = lib.ss_last_error(None).decode()
        if st == 0:
            lib.spin_system_destroy(h)
        return st, msg

    bad_col = lat.col.copy()
    bad_col[4] = 1000
    self_col = lat.col.copy()
    self_col[0] = 0
    bad_rp = lat.row_ptr.copy()
    bad_rp[5] = bad_rp[4] - 1
    asym = lat.J.copy()
    asym[0] *= 2
    cases = [
        (dict(col=bad_col), "out of range"),
        (dict(col=self_col), "self bond"),
        (dict(row_ptr=bad_rp), "decreases"),
        (dict(dt=0.0), "dt"),
        (dict(alpha=-0.1), "alpha"),
        (dict(T=-1.0), "T must"),
        (dict(mu_s=np.zeros(lat.n)), "mu_s"),
        (dict(J=np.full(lat.nnz, np.nan)), "not finite"),
        (dict(n=0), "out of range"),
    ]
    for over, text in cases:
        st, msg = create(**over)
        assert st == 1, (over, st, msg)  # SS_ERR_INVALID_ARG
        assert text in msg, (over, msg)


def test_binding_rejects_mismatched_per_system_arguments(lib):
    """The Python front end checks per-system argument counts before it calls the library."""
    from paper_1310_6143_gb300 import lattice as L
    from paper_1310_6143_gb300.system import SpinSystem

    lats = [L.simple_cubic(3, 3, 3)] * 2
    with pytest.raises(ValueError, match="S0"):
        SpinSystem(lats, S0=[L.random_state(27, 1)])
    with pytest.raises(ValueError, match="T"):
        SpinSystem(lats, T=[1.0, 2.0, 3.0])
    with pytest.raises(ValueError, match="precision"):
        SpinSystem(lats[0], precision="bf16")

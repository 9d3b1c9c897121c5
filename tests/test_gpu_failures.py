"""Failure handling with device-memory exhaustion injected on the host (no GPU fault): every
device allocation of a create, of the demagnetising-field set-up and of the Monte Carlo
set-up is made to fail in turn.  The call returns SS_ERR_OOM, a failed create holds no device
memory, a handle whose allocation failed reports SS_ERR_STATE afterwards, and destroying it
releases everything."""
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1310_6143_gb300 import _binding as B
    from paper_1310_6143_gb300.system import SpinSystem

    lib = B.load()
    yield lib, SpinSystem, B.SpinSysError
    lib.ss_debug_fail_allocations(-1)


def _lat():
    return L.simple_cubic(6, 6, 6, periodic=(False, False, False), J=6e-21, k_u=1e-23, with_pos=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_allocation_of_create_can_fail(env, precision):
    lib, SS, Err = env
    base = lib.ss_debug_live_bytes()
    needed = None
    try:
        for k in range(200):
            lib.ss_debug_fail_allocations(k)
            try:
                s = SS(_lat(), T=300.0, precision=precision)
            except Err as e:
                assert "OOM" in str(e)
                assert lib.ss_debug_live_bytes() == base  # nothing left behind
                continue
            lib.ss_debug_fail_allocations(-1)
            s.step(3)  # the handle created with exactly k allocations works
            s.close()
            needed = k
            break
    finally:
        lib.ss_debug_fail_allocations(-1)
    assert needed is not None and needed > 10
    assert lib.ss_debug_live_bytes() == base


@pytest.mark.parametrize("what", ["demag", "mc"])
def test_allocation_failure_after_create(env, what):
    lib, SS, Err = env
    base = lib.ss_debug_live_bytes()
    a = 3e-10
    try:
        for k in range(100):
            with SS(_lat(), T=300.0, precision="fp64") as s:
                held = lib.ss_debug_live_bytes()
                lib.ss_debug_fail_allocations(k)
                try:
                    if what == "demag":
                        s.set_demag(2 * a, a ** 3)
                    else:
                        s.mc_step(1)
                    failed = False
                except Err as e:
                    assert "OOM" in str(e)
                    failed = True
                lib.ss_debug_fail_allocations(-1)
                if not failed:
                    s.step(2)
                    break
                assert lib.ss_debug_live_bytes() >= held
                with pytest.raises(Err, match="STATE"):
                    s.step(1)
            assert lib.ss_debug_live_bytes() == base
        else:
            pytest.fail("the set-up never succeeded")
    finally:
        lib.ss_debug_fail_allocations(-1)
    assert lib.ss_debug_live_bytes() == base

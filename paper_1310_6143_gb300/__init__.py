"""GB300-native stochastic Heun-LLG atomistic spin dynamics (arXiv:1310.6143 hot path).

* ``lattice``  -- seeded synthetic systems (CSR neighbour lists, moments, anisotropy).
* ``SpinSystem`` -- one handle of the C-ABI library libspinsys.so (CUDA, sm_103a).
* ``build``    -- compiles the library in-tree with nvcc.

Importing the package does not load the CUDA library; the first ``SpinSystem`` does, and
fails loudly if it is missing.
"""
from . import lattice  # noqa: F401


def __getattr__(name):
    if name in ("SpinSystem", "debug_philox", "debug_gaussians"):
        from . import system

        return getattr(system, name)
    raise AttributeError(name)

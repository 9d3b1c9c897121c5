"""FP64 CPU oracle of the stochastic Heun-LLG step (with the optional macrocell
demagnetising field) and of the Hinzke-Nowak Monte Carlo step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product package never imports it, and the oracle shares
no code with the CUDA path.
"""
from .oracle import (  # noqa: F401
    FLAGS,
    OracleSystem,
    build,
    lib_path,
    philox4x32_10,
    philox_bulk,
    gaussians_bulk,
    thermal_gaussians,
    init_sphere,
    fields,
    moment_energy,
    heun_run,
    midpoint_run,
    sib_run,
    set_threads,
    max_threads,
    colour_greedy,
    mc_sigma_g,
    mc_run,
    macrocells,
    demag_fields,
)

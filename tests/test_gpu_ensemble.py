"""FP32-mixed against FP64 at equilibrium: |M|/Ms of the FP32-mixed ensemble lies within
3 standard errors of the FP64 ensemble.

Each ensemble is one batched handle of 8 independent copies (different seeds) of an fcc
ferromagnet shaped like the 64^3-cell workload but 16^3 cells (J = 11.2e-21 J,
mu_s = 1.72 muB, k_u = 6.69e-24 J || z, alpha = 0.05, dt = 1e-16 s), started ordered and
held at 1500 K (the top of the workload's sweep).  Per copy, |m| is averaged over the last
4000 of 7000 steps from the per-step record; the ensembles are compared by their means.
"""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


def _ensemble(precision, seeds, T=1500.0, equil=3000, avg=4000):
    from paper_1310_6143_gb300.system import SpinSystem

    lat = L.fcc(16, 16, 16, J=11.2e-21, k_u=6.69e-24)
    lats = [lat] * len(seeds)
    with SpinSystem(lats, alpha=0.05, dt=1e-16, T=T, seed=seeds, sys_id=list(range(len(seeds))),
                    precision=precision) as s:
        s.step(equil)
        cap = s.info()["record_capacity"]
        ms = []
        done = 0
        while done < avg:
            k = min(cap, avg - done)
            first = s.step_index
            s.step(k)
            rec = s.record(first, k)  # (k, systems, 8)
            ms.append(np.linalg.norm(rec[:, :, :3], axis=2) / rec[:, :, 3])
            done += k
    m = np.concatenate(ms, axis=0)  # (avg, systems)
    return m.mean(axis=0)


def test_fp32_mixed_equilibrium_magnetisation_within_3_sigma_of_fp64():
    seeds = [101, 202, 303, 404, 505, 606, 707, 808]
    m64 = _ensemble("fp64", seeds)
    m32 = _ensemble("fp32", [s + 1 for s in seeds])
    se = np.sqrt(m64.var(ddof=1) / m64.size + m32.var(ddof=1) / m32.size)
    assert 0.3 < m64.mean() < 0.95  # ordered, well below saturation at 1500 K
    assert abs(m32.mean() - m64.mean()) <= 3 * se, (m32.mean(), m64.mean(), se)

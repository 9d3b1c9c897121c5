"""FP32-mixed against FP64 at equilibrium on the full fcc 64^3-cell workload (1,048,576 spins,
J = 11.2e-21 J, mu_s = 1.72 muB, k_u = 6.69e-24 J || z, alpha = 0.05, dt = 1e-16 s) at three
temperatures of its 0-1500 K sweep.

Each ensemble is one batched handle of eight independent copies (different seeds), started
ordered; per copy |m| is averaged over six blocks of 500 steps after 3000 steps of
equilibration (per-step record), and the FP32-mixed ensemble mean of these 48 block means
must lie within 3 combined standard errors of the FP64 one.
With SPINSYS_REPORT_DIR set, the table of means and standard errors is written there as JSON.
"""
import json
import os

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu

SEEDS = [11, 22, 33, 44, 55, 66, 77, 88]
BLOCKS, BLOCK = 6, 500


def _ensemble(precision, seeds, T, equil=3000):
    from paper_1310_6143_gb300.system import SpinSystem

    lat = L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24)
    with SpinSystem([lat] * len(seeds), alpha=0.05, dt=1e-16, T=T, seed=seeds, sys_id=list(range(len(seeds))),
                    precision=precision) as s:
        s.step(equil)
        assert s.info()["record_capacity"] >= BLOCK
        blocks = []
        for _ in range(BLOCKS):
            first = s.step_index
            s.step(BLOCK)
            rec = s.record(first, BLOCK)  # (steps, systems, 8)
            blocks.append((np.linalg.norm(rec[:, :, :3], axis=2) / rec[:, :, 3]).mean(axis=0))
    return np.concatenate(blocks)  # block means of every copy


@pytest.mark.parametrize("T", [300.0, 900.0, 1500.0])
def test_fcc64_fp32_mixed_equilibrium_within_3_sigma_of_fp64(T):
    m64 = _ensemble("fp64", SEEDS, T)
    m32 = _ensemble("fp32", [s + 100 for s in SEEDS], T)
    se = float(np.sqrt(m64.var(ddof=1) / m64.size + m32.var(ddof=1) / m32.size))
    out = os.environ.get("SPINSYS_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"fcc64_equilibrium_{int(T)}K.json"), "w") as f:
            json.dump({"T_K": T, "m_fp64": float(m64.mean()), "m_fp32": float(m32.mean()),
                       "se_fp64": float(m64.std(ddof=1) / np.sqrt(m64.size)),
                       "se_fp32": float(m32.std(ddof=1) / np.sqrt(m32.size)), "se_combined": se,
                       "copies": len(SEEDS), "blocks_per_copy": BLOCKS, "block_steps": BLOCK}, f)
    assert 0.3 < m64.mean() < 1.0
    assert abs(m32.mean() - m64.mean()) <= 3 * se, (m32.mean(), m64.mean(), se)

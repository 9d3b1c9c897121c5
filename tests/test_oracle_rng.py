"""Pins of the oracle's counter-based generator and Gaussian transform.

Philox4x32-10 is checked against an independent implementation (the header-only
``at::philox_engine`` shipped with PyTorch, compiled here with g++), and both the uniform
words and the Box-Muller Gaussians are checked statistically.  No known-answer vectors are
typed in from memory.
"""
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _torch_philox_binary(tmp_path_factory):
    import torch

    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch's Philox header is not installed")
    d = tmp_path_factory.mktemp("philox")
    src = d / "p.cpp"
    src.write_text(
        "#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\n#include <cstdlib>\n"
        "int main(int c, char** v){ unsigned long long seed=strtoull(v[1],0,0), sub=strtoull(v[2],0,0),"
        " off=strtoull(v[3],0,0); at::philox_engine e(seed, sub, off);"
        " for(int i=0;i<4;i++) printf(\"%u \", e()); printf(\"\\n\"); return 0; }\n")
    exe = d / "p"
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}", "-o", str(exe), str(src)], check=True)
    return str(exe)


def test_philox_matches_independent_implementation(oracle_mod, tmp_path_factory):
    """torch's engine uses counter (offset lo, offset hi, subsequence lo, subsequence hi)
    and key (seed lo, seed hi): the same published Philox4x32-10 block function."""
    exe = _torch_philox_binary(tmp_path_factory)
    rng = np.random.default_rng(7)
    cases = [(0, 0, 0), (1, 0, 0), (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF)]
    cases += [tuple(int(v) for v in rng.integers(0, 2 ** 63, size=3)) for _ in range(20)]
    for seed, sub, off in cases:
        out = subprocess.run([exe, str(seed), str(sub), str(off)], check=True, capture_output=True,
                             text=True).stdout.split()
        ref = np.array([int(v) for v in out], dtype=np.uint32)
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        np.testing.assert_array_equal(oracle_mod.philox4x32_10(ctr, key), ref)


def test_philox_uniform_words(oracle_mod):
    w = oracle_mod.philox_bulk([0, 17, 3, 0], [12345, 678], 250_000).ravel()
    # chi-square on 256 bins of the top byte and of the low byte
    for bits in (w >> 24, w & 0xFF):
        counts = np.bincount(bits.astype(np.int64), minlength=256)
        chi2, p = stats.chisquare(counts)
        assert p > 1e-4, p
    # bit balance
    bits = np.unpackbits(w.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 5e-4
    # consecutive counters are uncorrelated
    u = (w.astype(np.float64) + 0.5) / 2 ** 32
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5e-3


def test_philox_key_and_counter_sensitivity(oracle_mod):
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        diff = np.unpackbits((oracle_mod.philox4x32_10(c, [5, 6]) ^ base).view(np.uint8)).sum()
        assert 40 < diff < 88  # about half of 128 bits flip
    diff = np.unpackbits((oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 7]) ^ base).view(np.uint8)).sum()
    assert 40 < diff < 88


def test_thermal_gaussians_are_standard_normal(oracle_mod):
    g = oracle_mod.gaussians_bulk(seed=99, sys_id=3, step=11, n=200_000)
    for c in range(3):
        x = g[:, c]
        assert abs(x.mean()) < 0.015
        assert abs(x.var() - 1) < 0.015
        assert abs(stats.kurtosis(x, fisher=False) - 3) < 0.06
        assert stats.kstest(x, "norm").pvalue > 1e-4
    # components independent
    c = np.corrcoef(g.T)
    assert np.abs(c - np.eye(3)).max() < 0.01
    # |g|^2 is chi-square with 3 degrees of freedom
    assert stats.kstest((g * g).sum(1), "chi2", args=(3,)).pvalue > 1e-4


def test_thermal_gaussians_depend_on_every_counter_field(oracle_mod):
    a = oracle_mod.thermal_gaussians(5, 0, 10, 20)
    for args in ((6, 0, 10, 20), (5, 1, 10, 20), (5, 0, 11, 20), (5, 0, 10, 21), (5 + (1 << 32), 0, 10, 20)):
        assert np.abs(oracle_mod.thermal_gaussians(*args) - a).max() > 1e-6
    # bulk and single-spin paths agree
    bulk = oracle_mod.gaussians_bulk(5, 0, 20, 12)
    np.testing.assert_array_equal(bulk[10], a)


def test_init_sphere_uniform(oracle_mod):
    S = oracle_mod.init_sphere(2, 0, 100_000)
    np.testing.assert_allclose(np.linalg.norm(S, axis=1), 1.0, atol=1e-15)
    assert np.abs(S.mean(0)).max() < 0.01
    # uniform on the sphere: each component is uniform on [-1, 1]
    for c in range(3):
        assert stats.kstest(S[:, c], "uniform", args=(-1, 2)).pvalue > 1e-4

"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes per Heun pass and per
spin-step, the bytes of the implemented layout, the timed window around the temperature
pulse, and the clock-record summary (samples kept only inside the timed window, throttle
reasons)."""
import datetime
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("z,p,expect", [(6.0, 4, 176.0), (6.0, 8, 296.0), (12.0, 4, 272.0), (12.0, 8, 440.0),
                                        (5.875, 4, 174.0), (5.875, 8, 293.0)])
def test_step_bytes_per_spin(z, p, expect):
    # state: read S, write S' and P, read them back, write S (6 vectors of 3 words); CSR
    # columns, values and the row offset once per field evaluation
    assert bench.step_bytes_per_spin(p, z) == pytest.approx(expect)
    assert bench.step_bytes_per_spin(p, z) == pytest.approx(6 * 3 * p + 2 * (z * (4 + p) + 4))


def test_pass_and_layout_bytes():
    # one Heun pass of the film: 9 words and the CSR row; the step is two passes
    assert bench.pass_bytes_per_spin(4, 5.875) == pytest.approx(87.0)
    assert bench.step_bytes_per_spin(4, 5.875) == pytest.approx(2 * bench.pass_bytes_per_spin(4, 5.875))
    # the implemented layout: 24 words of state, half the Gaussians drawn ahead (written and
    # read back), one pattern byte per pass, a single material (no index)
    assert bench.layout_bytes_per_spin(4, 5.875, 0.5, True, patterns=True, one_material=True) == pytest.approx(
        96 + 12 + 2)
    # the CSR and the material index instead
    assert bench.layout_bytes_per_spin(4, 5.875, 0.5, True) == pytest.approx(96 + 12 + 2 * (5.875 * 4 + 4) + 8)
    assert bench.layout_bytes_per_spin(8, 6, 0.0, False) == pytest.approx(192 + 2 * (6 * 4 + 4) + 2 * 6 * 8 + 8)


def test_timed_window_is_centred_on_the_pulse():
    for steps, warmup in ((1000, 10), (20, 5), (3, 3)):
        first = bench.timed_window(steps, warmup) + warmup
        assert first <= bench.PULSE_PEAK_STEP < first + steps
    assert bench.timed_window(30000, 10) == 0


def test_pulse_peak_and_width():
    dt = 1e-16
    T = bench.pulse_T(20001, dt=dt)
    k0 = int(round(1e-12 / dt))
    assert T[k0] == pytest.approx(1200.0)
    assert T[0] == pytest.approx(300.0, abs=1e-6)
    half = int(round(50e-15 / dt))  # FWHM 100 fs: half the excursion at t0 +- 50 fs
    assert T[k0 + half] == pytest.approx(750.0, rel=1e-9)
    assert T[k0 - half] == pytest.approx(750.0, rel=1e-9)


def _row(t, sm, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join(["0", str(sm), "2070", "900.0", "0x0", *reasons, stamp])


def test_clock_summary_keeps_the_timed_window(tmp_path):
    t = 1.7e9
    path = tmp_path / "clocks.csv"
    rows = [_row(t - 0.3, 600), _row(t + 0.1, 2070), _row(t + 0.2, 2055), _row(t + 0.3, 2070),
            _row(t + 2.0, 1200, ("Not Active", "Not Active", "Not Active", "Active"))]
    path.write_text("\n".join(rows) + "\n")
    ck = bench.Clocks(str(path))
    every = ck.summary()
    assert every["samples"] == 5 and every["reasons"] == ["sw_power_cap"]
    ck.mark(t, t + 1.0)
    inside = ck.summary()
    assert inside == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_clock_summary_without_samples(tmp_path):
    ck = bench.Clocks(str(tmp_path / "absent.csv"))
    assert ck.summary()["reasons"] == ["unsampled"]
    assert bench._smi_time("not a time") == -1.0

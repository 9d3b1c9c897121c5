"""Benchmark: stochastic Heun-LLG spin-steps/s on one GB300 (and N independent replicas).

Default workload: the 1024 x 1024 x 16 simple-cubic thin film (16,777,216 spins, in-plane
periodic, free z surfaces, J = 6.0e-21 J, mu_s = 1.5 muB, k_u = 1.0e-24 J || z,
alpha = 0.02, dt = 1e-16 s) under the 100 fs Gaussian temperature pulse (1200 K peak on a
300 K base, centred at 1 ps), FP32-mixed precision.  A step is one full Heun step of the
whole film: thermal field, predictor, corrector, renormalisation and the FP64 moment and
energy reductions.  The state (~0.8 GB of working arrays) is far larger than L2, so no
flush is needed between steps.

Also reported: the same film in plain FP64, and the 256-grain batched ensemble in one
handle (FP32-mixed, launch shape picked by the autotuner).  The CPU oracle (FP64, all host cores) is timed on a
bounded sample of the film for the CPU baseline.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torchrun each
rank advances its own replica of the film (statistical parallelism, no collective).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LLG spin-steps/s on 1 GB300 (FP32 vs FP64 Heun); % of HBM roofline"
KB = 1.3807e-23


def pulse_T(nsteps, dt=1e-16, base=300.0, peak=1200.0, t0=1e-12, fwhm=100e-15):
    """Gaussian temperature pulse: base + (peak - base) exp(-(t - t0)^2 / (2 s^2)), FWHM 100 fs."""
    s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    t = np.arange(nsteps) * dt
    return base + (peak - base) * np.exp(-((t - t0) ** 2) / (2 * s * s))


# Algorithmic HBM bytes per spin of one Heun pass with the CSR as stored: the pass reads one
# spin vector and writes two (predictor: S -> S', P) or reads two and writes one (corrector:
# S', P -> S), 9 words, and reads the CSR row once (z columns and values, one row offset):
# 9 p + z (4 + p) + 4.  The step is two passes: 18 p + 2 (z (4 + p) + 4), for the film (mean
# z = 5.875) 87 B per pass and 174 B per step in FP32, 146.5 and 293 B in FP64.
def pass_bytes_per_spin(real_bytes, nnz_per_spin):
    return 9 * real_bytes + nnz_per_spin * (4 + real_bytes) + 4


def step_bytes_per_spin(real_bytes, nnz_per_spin):
    return 2 * pass_bytes_per_spin(real_bytes, nnz_per_spin)


# Bytes the implemented layout moves per spin-step: S, S', the half step Q and the stored
# thermal field (24 words), the Gaussians drawn ahead (written and read back for a fraction
# f of the spins), the neighbour rows once per pass -- one byte per spin with row patterns,
# else the CSR columns and row offset (and J unless every bond has the same J_ij/mu_s,i) --
# and the material index once per pass unless the handle has a single material.
def layout_bytes_per_spin(real_bytes, nnz_per_spin, f_ahead, j_uniform, patterns=False, one_material=False):
    rows = 2.0 if patterns else 2 * (nnz_per_spin * 4 + 4) + (0 if j_uniform else 2 * nnz_per_spin * real_bytes)
    return 24 * real_bytes + 6 * real_bytes * f_ahead + rows + (0 if one_material else 8)


# The FP64 form's step kernels run every operation on the FP64 pipe (2 instructions per cycle
# per SM on GB300): FP64 instructions per spin counted by ncu (sass_thread_inst_executed_op_
# dadd/dmul/dfma) on the film's predictor, profiles/k_predictor_film1024x1024x16_fp64.md.
# Each counts as 2 flop-equivalents, the convention of the chip's FP64 rating.
FP64_FORM_PREDICTOR_FP64_PER_SPIN = 102.0

# DRAM bytes per launch of the default film shape (block, tile, draw-ahead eighths), read from
# one ncu capture of the FP32-mixed kernels (profiles/k_predictor_film1024x1024x16_fp32.md,
# profiles/k_corrector_film1024x1024x16_fp32.md), not measured in this run.
DEFAULT_FILM_SHAPE = (512, 4096, 4)
KERNEL_DRAM_BYTES = {"k_predictor": 0.902e9, "k_corrector": 0.897e9}
SMS = 152
NO_AUTOTUNE = False
EXEC_NAMES = {0: "auto", 1: "kernels", 2: "graph", 3: "persistent", 4: "system_blocks", 5: "cluster"}
FP64_SLOTS_PER_SM_CYCLE = 2
PULSE_PEAK_STEP = 10_000  # the temperature pulse peaks at t0 = 1 ps = step 10,000 at dt = 1e-16 s


def timed_window(steps, warmup):
    """First step of the warm-up so that the timed steps are centred on the pulse peak."""
    return max(0, PULSE_PEAK_STEP - steps // 2 - warmup)


def _smi_time(stamp):
    """nvidia-smi's timestamp ('2026/12/03 10:00:00.123') as host epoch seconds; -1 if unreadable."""
    try:
        return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return -1.0


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None
        self.window = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # the sampler is producing rows before the timed region starts
        except Exception:
            self.proc = None
        return self

    def mark(self, t0, t1):
        """Host wall-clock bounds of the timed region: only the samples inside it are summarised."""
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index=0):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 10 and r[0].strip() == str(device_index)]
        if self.window:
            inside = [r for r in rows if self.window[0] <= _smi_time(r[9]) <= self.window[1]]
            rows = inside or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(lat, T, seconds=15.0):
    """The FP64 oracle, as it stands, on the host cores: one film step (or more to fill
    about `seconds`) from the all-up state."""
    import oracle as O

    O.build()
    threads = O.max_threads()
    O.set_threads(threads)
    ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.02, dt=1e-16,
                         seed=5)
    S = np.ascontiguousarray(np.broadcast_to([0.0, 0.0, 1.0], (lat.n, 3)))
    t0 = time.perf_counter()
    S, _ = O.heun_run(ref, S, 1, T[:1], record=True)
    one = time.perf_counter() - t0
    steps = 1
    extra = int(max(0, min(9, seconds / max(one, 1e-3) - 1)))
    if extra:
        t1 = time.perf_counter()
        S, _ = O.heun_run(ref, S, extra, T[1:1 + extra], step0=1, record=True)
        one = (one + time.perf_counter() - t1)
        steps += extra
    # one more step on a single thread
    O.set_threads(1)
    t2 = time.perf_counter()
    S, _ = O.heun_run(ref, S, 1, T[steps:steps + 1], step0=steps, record=True)
    single = time.perf_counter() - t2
    O.set_threads(threads)
    return {"value": lat.n * steps / one, "unit": "spin-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} Heun step(s) of the full 1024x1024x16 film (FP64, with per-step moment/energy "
                      f"record), {one:.1f} s, oracle built gcc {' '.join(O.FLAGS)}",
            "single_thread_value": lat.n / single, "cpu_model": cpu_model(), "build": "gcc " + " ".join(O.FLAGS)}


def fp32_error(stream):
    """The FP32-mixed form's trajectory error against the FP64 oracle, as numbers: every spin of
    the film after eight benchmarked steps (a pulse-shaped schedule, random start), and the sc
    10^3 workload after 100 steps (the stated 1e-4 tolerance is for 100 steps), with the FP64
    form beside each (1e-12 after 1000 steps for sc 10^3)."""
    import oracle as O
    from paper_1310_6143_gb300 import lattice as L
    from paper_1310_6143_gb300.system import SpinSystem

    O.build()
    O.set_threads(O.max_threads())

    def run(lat, precision, steps, T, S0, alpha, seed):
        with SpinSystem(lat, alpha=alpha, dt=1e-16, T=0.0, seed=seed, S0=S0, precision=precision,
                        stream=stream) as s:
            s.set_temperature_schedule(T)
            start = s.spins()
            s.step(steps)
            return start, s.spins(), s.record(0, steps)[:, 0, :]

    def oracle_run(lat, start, steps, T, alpha, seed):
        ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=alpha, dt=1e-16,
                             seed=seed)
        return O.heun_run(ref, start, steps, T, record=True)

    out = {}
    film = L.film(1024, 1024, 16)
    T8 = np.array([300.0, 450.0, 700.0, 1000.0, 1200.0, 1000.0, 700.0, 450.0])
    S0 = L.random_state(film.n, 31)
    for prec in ("fp32", "fp64"):
        start, S, rec = run(film, prec, 8, T8, S0, 0.02, 5)
        S_ref, rec_ref = oracle_run(film, start, 8, T8, 0.02, 5)
        out[f"film_8_steps_{prec}"] = {"max_abs_dS": float(np.abs(S - S_ref).max()),
                                       "max_rel_dM": float(np.abs(rec[:, :3] - rec_ref[:, :3]).max() / rec_ref[0, 3])}
    sc = L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24)
    for prec, steps in (("fp32", 100), ("fp64", 1000)):
        start, S, rec = run(sc, prec, steps, np.full(steps, 300.0), L.uniform_state(sc.n), 0.1, 1)
        S_ref, rec_ref = oracle_run(sc, start, steps, np.full(steps, 300.0), 0.1, 1)
        out[f"sc10_{steps}_steps_{prec}"] = {"max_abs_dS": float(np.abs(S - S_ref).max()),
                                              "max_rel_dM": float(np.abs(rec[:, :3] - rec_ref[:, :3]).max()
                                                                  / rec_ref[0, 3])}
    out["tolerances"] = {"fp32_100_steps": 1e-4, "fp64_1000_steps": 1e-12}
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def time_workload(lats, kw, precision, steps, stream, warmup=5, autotune=True):
    autotune = autotune and not NO_AUTOTUNE
    """spin-steps/s of `steps` Heun steps on one handle (CUDA events on its stream)."""
    import torch

    from paper_1310_6143_gb300.system import SpinSystem

    n = sum(l.n for l in (lats if isinstance(lats, list) else [lats]))
    with SpinSystem(lats, precision=precision, stream=stream, **kw) as s:
        info = s.autotune(8) if autotune else s.info()
        s.step(warmup)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        s.sync()
        ms = e0.elapsed_time(e1)
    return {"value": n * steps / (ms * 1e-3), "ms_per_step": ms / steps, "steps": steps,
            "exec": EXEC_NAMES[info["exec"]], "block": info["block"],
            "tile": info["tile"]}


def workload_table(stream, rank):
    """The five workload shapes of the method's benchmark set, FP32-mixed and FP64."""
    from paper_1310_6143_gb300 import lattice as L

    rows = {}
    sc = L.simple_cubic(10, 10, 10, J=6.0e-21, k_u=1.0e-24)
    for prec in ("fp64", "fp32"):
        rows[f"sc10_{prec}"] = dict(spins=sc.n, **time_workload(sc, dict(alpha=0.1, dt=1e-16, T=300.0, seed=1 + rank),
                                                                 prec, 2000, stream))
    fcc = L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24)
    kw = dict(alpha=0.05, dt=1e-16, T=1000.0, seed=2 + rank, init_random=True)
    for prec, k in (("fp32", 200), ("fp64", 50)):
        rows[f"fcc64_{prec}"] = dict(spins=fcc.n, **time_workload(fcc, kw, prec, k, stream))
    # a temperature sweep as one batch: 1,024 independent 10^3 lattices from 0 to 1,023 K
    sweep = [sc] * 1024
    rows["sc10_x1024_sweep_fp32"] = dict(spins=sc.n * 1024, systems=1024, **time_workload(
        sweep, dict(alpha=0.1, dt=1e-16, T=[float(t) for t in range(1024)], seed=1 + rank,
                    sys_id=list(range(1024))), "fp32", 500, stream))
    # tensorial exchange: the fcc crystal with an interface-type DM term (|D| = 0.1 J) and
    # cubic anisotropy, 9 exchange values per bond
    dm = L.with_dm(L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24, with_pos=True), D=1.12e-21)
    dm.k_c = np.full(dm.n, 5e-24)
    kw = dict(alpha=0.05, dt=1e-16, T=300.0, seed=4 + rank, init_random=True)
    for prec, k in (("fp32", 200), ("fp64", 50)):
        rows[f"fcc64_dm_cubic_{prec}"] = dict(spins=dm.n, **time_workload(dm, kw, prec, k, stream))
    cs = L.core_shell_sphere()
    kw = dict(alpha=0.1, dt=1e-16, T=10.0, H=(1.0, 0.0, 0.0), seed=3 + rank)
    for prec, k in (("fp32", 400), ("fp64", 100)):
        rows[f"core_shell_{prec}"] = dict(spins=cs.n, **time_workload(cs, kw, prec, k, stream))
    return rows


def time_mc(lat, kw, precision, steps, stream, warmup=3, rows="auto"):
    """Hinzke-Nowak Monte Carlo steps (one trial move per spin each, with the per-step
    moment/energy record), timed with CUDA events on the handle's stream."""
    import torch
    from paper_1310_6143_gb300.system import SpinSystem

    with SpinSystem(lat, precision=precision, stream=stream, **kw) as s:
        if rows != "auto":
            s.set_exchange_rows(rows)
        s.mc_step(warmup)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.mc_step(steps)
        e1.record(stream)
        e1.synchronize()
        s.sync()
        ms = e0.elapsed_time(e1)
        acc, tried = s.mc_stats(0)
    return {"value": lat.n * steps / (ms * 1e-3), "unit": "spin trial moves/s", "steps": steps,
            "ms_per_step": ms / steps, "acceptance": acc / tried}


def mc_table(stream, rank, film_steps=100):
    """Monte Carlo legs: the film (16.8 M spins, two colours) and the paper's Fig. MCLLG
    system (simple cubic 28^3, J = 6.0e-21 J/link, periodic) at 300 K."""
    from paper_1310_6143_gb300 import lattice as L

    rows = {}
    film = L.film(1024, 1024, 16)
    for prec, k in (("fp32", film_steps), ("fp64", max(10, film_steps // 4))):
        rows[f"film_{prec}"] = dict(spins=film.n, **time_mc(film, dict(T=300.0, seed=7 + rank), prec, k, stream))
    sc28 = L.simple_cubic(28, 28, 28, J=6.0e-21, k_u=0.0)
    for prec in ("fp32", "fp64"):
        rows[f"sc28_{prec}"] = dict(spins=sc28.n, **time_mc(sc28, dict(T=300.0, seed=31 + rank), prec, 1000, stream))
    return rows


def demag_table(stream, rank):
    """Macrocell demagnetising field on the paper's ellipsoid: cost of one field update
    (cell-pair interactions per second) and Heun-LLG throughput with the paper's update
    every 100 steps."""
    import torch
    from paper_1310_6143_gb300.system import SpinSystem

    from paper_1310_6143_gb300 import lattice as L

    lat = L.prolate_ellipsoid()
    vatom, cell = lat.meta["atom_volume"], 2 * lat.meta["a"]
    grid = np.floor((lat.pos - lat.pos.min(axis=0)) / cell).astype(np.int64)
    nc = int(np.unique(grid[:, 0] + 4096 * (grid[:, 1] + 4096 * grid[:, 2])).size)
    rows = {}
    for prec in ("fp32", "fp64"):
        res = {}
        for every in (0, 1, 100):
            with SpinSystem(lat, alpha=0.1, dt=1e-16, T=300.0, seed=9 + rank, precision=prec,
                            stream=stream) as s:
                s.set_exec("kernels")
                if every:
                    s.set_demag(cell, vatom, every)
                s.step(5)
                s.sync()
                k = 400
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(k)
                e1.record(stream)
                e1.synchronize()
                s.sync()
                res[every] = e0.elapsed_time(e1) / k
        upd = max(res[1] - res[0], 1e-9)
        rows[f"ellipsoid_{prec}"] = {"spins": lat.n, "macrocells": nc, "update_ms": upd,
                                     "cell_pairs_per_s": nc * (nc - 1) / (upd * 1e-3),
                                     "ms_per_step_no_demag": res[0], "ms_per_step_every_100": res[100],
                                     "value": lat.n / (res[100] * 1e-3), "unit": "spin-steps/s (update every 100)"}
    return rows


def long_range_table(stream, rank, cells=64, steps=20, hbm_peak=6800.0):
    """Long exchange rows: fcc with exchange to 4a (1,060 neighbours per atom, 30 shells), the
    shape of the paper's long-ranged exchange runs (over 1,000 neighbours, ~1.6e6 atoms),
    at 300 K.  Heun throughput with a warp per row (packed bond words) and with a thread per
    row, and the warp-per-row exchange pass alone against the DRAM roofline (its algorithmic
    bytes: the 4-byte bond words, row pointers, material indices, the spins once and the field
    written) and, in FP64, against the FP64 pipe (three FMAs per bond)."""
    import torch
    from paper_1310_6143_gb300.system import SpinSystem

    from paper_1310_6143_gb300 import lattice as L

    lat = L.fcc_long_range(cells, cells, cells, r_cut=4.0)
    n, nnz = lat.n, lat.nnz
    rows = {}
    for prec, k in (("fp32", steps), ("fp64", max(4, steps // 4))):
        rs = 4 if prec == "fp32" else 8
        for mode in ("warp", "thread"):
            with SpinSystem(lat, alpha=0.1, dt=1e-16, T=300.0, seed=11 + rank, precision=prec,
                            stream=stream) as s:
                s.set_exchange_rows("auto" if mode == "warp" else "thread")
                info = s.info()
                s.step(3)
                s.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(k)
                e1.record(stream)
                e1.synchronize()
                s.sync()
                ms = e0.elapsed_time(e1) / k
                row = {"spins": n, "bonds": nnz, "exchange_rows": info["exchange_rows"], "ms_per_step": ms,
                       "value": n / (ms * 1e-3), "unit": "spin-steps/s"}
                if mode == "warp":
                    t = s.time_rows(10)
                    alg = nnz * 4 + (n + 1) * 4 + n * 4 + 2 * 3 * n * rs
                    row.update(rows_pass_ms=t, rows_pass_bytes=alg, rows_pass_gbs=alg / (t * 1e-3) / 1e9,
                               rows_pass_hbm_frac=alg / (t * 1e-3) / 1e9 / hbm_peak,
                               rows_pass_fma_per_s=3 * nnz / (t * 1e-3),
                               rows_share_of_step=2 * t / ms)
            rows[f"fcc{cells}_lr_{prec}_{mode}"] = row
        # the semi-implicit scheme on the same rows (row passes before its predictor and corrector)
        with SpinSystem(lat, alpha=0.1, dt=1e-16, T=300.0, seed=11 + rank, precision=prec, stream=stream) as s:
            s.semi_implicit_step(3)
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.semi_implicit_step(k)
            e1.record(stream)
            e1.synchronize()
            s.sync()
            ms = e0.elapsed_time(e1) / k
        rows[f"fcc{cells}_lr_{prec}_semi_implicit"] = {"spins": n, "bonds": nnz, "ms_per_step": ms,
                                                        "value": n / (ms * 1e-3), "unit": "spin-steps/s"}
    # Monte Carlo on the same rows: a warp per 32 trials against a thread per trial (FP32-mixed)
    for mode in ("auto", "thread"):
        r = time_mc(lat, dict(T=300.0, seed=13 + rank), "fp32", 4, stream, warmup=1, rows=mode)
        rows[f"fcc{cells}_lr_fp32_mc_{'warp' if mode == 'auto' else 'thread'}"] = dict(spins=n, bonds=nnz, **r)
    return rows


def midpoint_table(stream, rank, steps=40):
    """The alternative integrators on the film at 300 K: the midpoint rule (fixed-point
    iterations from the Euler predictor, K = 3 and 4 per step) and the semi-implicit
    predictor-corrector, spin-steps/s and the largest |S| - 1 after the run."""
    import torch
    from paper_1310_6143_gb300.system import SpinSystem

    from paper_1310_6143_gb300 import lattice as L

    film = L.film(1024, 1024, 16)
    rows = {}
    for prec in ("fp32", "fp64"):
        for K in (3, 4):
            with SpinSystem(film, alpha=0.02, dt=1e-16, T=300.0, seed=5 + rank, precision=prec,
                            stream=stream) as s:
                s.midpoint_step(3, iterations=K)
                s.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.midpoint_step(steps, iterations=K)
                e1.record(stream)
                e1.synchronize()
                s.sync()
                ms = e0.elapsed_time(e1) / steps
                dev = float(np.abs(np.linalg.norm(s.spins(), axis=1) - 1).max())
            rows[f"film_{prec}_K{K}"] = {"spins": film.n, "iterations": K, "ms_per_step": ms,
                                         "value": film.n / (ms * 1e-3), "unit": "spin-steps/s",
                                         "max_length_error": dev}
        # the semi-implicit predictor-corrector (Mentink et al.'s scheme)
        with SpinSystem(film, alpha=0.02, dt=1e-16, T=300.0, seed=5 + rank, precision=prec, stream=stream) as s:
            s.semi_implicit_step(3)
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.semi_implicit_step(steps)
            e1.record(stream)
            e1.synchronize()
            s.sync()
            ms = e0.elapsed_time(e1) / steps
            dev = float(np.abs(np.linalg.norm(s.spins(), axis=1) - 1).max())
        rows[f"film_{prec}_semi_implicit"] = {"spins": film.n, "ms_per_step": ms, "value": film.n / (ms * 1e-3),
                                              "unit": "spin-steps/s", "max_length_error": dev}
    return rows


def run_reference(args):
    """The oracle arm: W untimed and K timed FP64 Heun steps of the oracle, as it stands, on the
    host cores.  Each step is one oracle step (with its moment/energy record) over a film of the
    benchmark's construction (1,024 sites wide, 16 thick, in-plane periodic, the same bonds per
    spin) whose depth is chosen from a one-step calibration so that all K + W steps take about
    two minutes; spin-steps/s is the film's spins x K over the timed steps' wall time."""
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_1310_6143_gb300 import lattice as L

    K, W = max(1, args.steps), max(0, args.warmup)
    O.build()
    threads = O.max_threads()
    O.set_threads(threads)

    def system(ny):
        lat = L.film(1024, ny, 16)
        ref = O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, alpha=0.02, dt=1e-16,
                             seed=5)
        return lat, ref, np.ascontiguousarray(np.broadcast_to([0.0, 0.0, 1.0], (lat.n, 3)))

    lat, ref, S = system(64)  # calibration, untimed
    t0 = time.perf_counter()
    O.heun_run(ref, S, 1, 300.0, record=True)
    rate = lat.n / max(time.perf_counter() - t0, 1e-6)
    ny = int(min(1024, max(8, 120.0 * rate / ((K + W) * 1024 * 16))))
    lat, ref, S = system(ny)
    T = pulse_T(K + W)
    if W:
        S, _ = O.heun_run(ref, S, W, T[:W], record=True)
    t0 = time.perf_counter()
    S, _ = O.heun_run(ref, S, K, T[W:], step0=W, record=True)
    secs = time.perf_counter() - t0
    v = lat.n * K / secs
    cb = {"value": v, "unit": "spin-steps/s", "cores": threads, "kind": "oracle",
          "sample": f"{K} Heun steps (after {W} untimed) of a 1024x{ny}x16 film of the workload's construction "
                    f"({lat.n} spins; FP64, with per-step moment/energy record), {secs:.1f} s, oracle built gcc "
                    f"{' '.join(O.FLAGS)}",
          "cpu_model": cpu_model(), "build": "gcc " + " ".join(O.FLAGS)}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "spin-steps/s", "n_gpus": 1,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * secs / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "film 1024x1024x16 sc, T pulse 300->1200 K, alpha 0.02, dt 1e-16 s",
                       "spins": 1024 * 1024 * 16, "sample_spins": lat.n, "nnz": int(lat.nnz)},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "spin-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, batched and CPU legs")
    ap.add_argument("--demag-only", action="store_true",
                    help="run only the demagnetising-field leg on the paper's ellipsoid and print it")
    ap.add_argument("--long-range-only", action="store_true",
                    help="run only the long-exchange-row leg (fcc, 1,060 neighbours per atom) and print it")
    ap.add_argument("--lr-cells", type=int, default=64,
                    help="cubic cells per axis of the long-exchange-row leg's fcc crystal (default 64: 1.05 M atoms)")
    ap.add_argument("--midpoint-only", action="store_true",
                    help="run only the midpoint-rule leg on the film and print it")
    ap.add_argument("--alt-steps", type=int, default=40,
                    help="timed steps of each alternative-integrator run with --midpoint-only")
    ap.add_argument("--mc-only", action="store_true",
                    help="run only a short Monte Carlo leg on the film (for profiling) and print it")
    ap.add_argument("--no-autotune", action="store_true", help="no autotuning in the batched and workload legs")
    ap.add_argument("--autotune-film", action="store_true",
                    help="autotune the film's launch shape too (default: the library's default shape, "
                         "whose ncu counters are in profiles/)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the headline film run (fp32 = FP32-mixed)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    global NO_AUTOTUNE
    NO_AUTOTUNE = args.no_autotune

    world, rank, local = dist_init()
    import torch

    torch.cuda.set_device(local)
    from paper_1310_6143_gb300 import lattice as L
    from paper_1310_6143_gb300.system import SpinSystem

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    lat = L.film(1024, 1024, 16)
    nnz_per = lat.nnz / lat.n
    # the timed steps are centred on the pulse peak (step 10,000): the schedule covers them
    step0 = timed_window(args.steps, args.warmup)
    total_steps = step0 + args.warmup + args.steps + 64
    T = pulse_T(total_steps + 16)
    stream = torch.cuda.Stream()
    res = {}
    if args.demag_only:
        if rank == 0:
            print(json.dumps({"demag": demag_table(stream, rank)}))
        return
    if args.long_range_only:
        if rank == 0:
            print(json.dumps({"long_range": long_range_table(stream, rank, cells=args.lr_cells, hbm_peak=hbm_peak)}))
        return
    if args.midpoint_only:
        if rank == 0:
            print(json.dumps({"midpoint": midpoint_table(stream, rank, steps=args.alt_steps)}))
        return
    if args.mc_only:
        film = dict(spins=lat.n, **time_mc(lat, dict(T=300.0, seed=7 + rank), args.precision, args.steps, stream,
                                           warmup=args.warmup))
        if rank == 0:
            print(json.dumps({"mc_film": film, "precision": args.precision}))
        return

    def timed_run(precision, steps, warmup, seed):
        with SpinSystem(lat, alpha=0.02, dt=1e-16, T=300.0, seed=seed + rank, sys_id=rank, precision=precision,
                        stream=stream) as s:
            s.set_temperature_schedule(T)
            info = s.autotune(6) if args.autotune_film else s.info()
            s.step_index = timed_window(steps, warmup)
            s.step(warmup)
            s.sync()
            first = s.step_index
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with Clocks(os.path.join(os.environ.get("SPINSYS_CLOCKS_DIR", tempfile.gettempdir()),
                                     f"clocks_{precision}.csv")) as ck:
                h0 = time.time()
                e0.record(stream)
                s.step(steps)
                e1.record(stream)
                e1.synchronize()
                ck.mark(h0, time.time())
            s.sync()
            torch.cuda.synchronize()
            barrier(world)
            ms = e0.elapsed_time(e1)
            ms = max_over_ranks(world, ms)
            kt = s.time_passes(5)
            # end to end through the public API: per step the temperature goes host->device,
            # the step runs, and the step's moment/energy record comes back device->host
            e2e_steps = max(5, min(steps, 50))
            s.set_exec("kernels")
            t0 = time.perf_counter()
            e2e_first = s.step_index
            for k in range(e2e_steps):
                s.set_temperature(float(T[(e2e_first + k) % len(T)]))
                s.step(1)
                s.record(e2e_first + k, 1)
            e2e_s = time.perf_counter() - t0
            mag = s.magnetisation()
        window = {"first_step": int(first), "steps": int(steps),
                  "T_min_K": float(T[first:first + steps].min()), "T_max_K": float(T[first:first + steps].max())}
        return ms, kt, e2e_s / e2e_steps, ck.summary(local), mag, info, window

    ms32, kt32, e2e32, clk32, mag32, info32, win32 = timed_run(args.precision, args.steps, args.warmup, 5)
    e2e32 = max_over_ranks(world, e2e32)  # the job's end-to-end step time: its slowest rank
    value = world * lat.n * args.steps / (ms32 * 1e-3)
    rb = 4 if args.precision == "fp32" else 8
    pass_b = pass_bytes_per_spin(rb, nnz_per)
    step_b = step_bytes_per_spin(rb, nnz_per)
    # the dominant kernel of the step, by live CUDA-event time on the handle's stream
    dom = "k_predictor" if kt32["predictor_ms"] >= kt32["corrector_ms"] else "k_corrector"
    dom_ms = kt32["predictor_ms"] if dom == "k_predictor" else kt32["corrector_ms"]
    kernel_gbs = pass_b * lat.n / (dom_ms * 1e-3) / 1e9
    step_gbs = step_b * lat.n / (ms32 / args.steps * 1e-3) / 1e9
    spt = info32["tile"] // info32["block"]
    f_ahead = ((info32["draw_ahead"] * spt) // 8) / spt if args.precision == "fp32" else 0.0
    j_rows = lat.J / np.repeat(lat.mu_s, np.diff(lat.row_ptr))
    lay_b = layout_bytes_per_spin(rb, nnz_per, f_ahead, bool(np.all(j_rows == j_rows[0])),
                                  patterns=info32.get("row_patterns", 0) > 0, one_material=info32["num_materials"] == 1)
    default_shape = (info32["block"], info32["tile"], info32["draw_ahead"]) == DEFAULT_FILM_SHAPE
    sm_ghz = (clk32.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))) / 1e3
    out = {
        "metric": METRIC, "value": value, "unit": "spin-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "film 1024x1024x16 sc (16,777,216 spins), in-plane periodic, J 6.0e-21, "
                               "k_u 1.0e-24 || z, alpha 0.02, dt 1e-16 s, T pulse 300->1200 K (100 fs FWHM, peak at "
                               f"step {PULSE_PEAK_STEP}); timed steps {win32['first_step']}..."
                               f"{win32['first_step'] + win32['steps'] - 1} of the schedule, centred on the pulse "
                               f"(T {win32['T_min_K']:.0f}-{win32['T_max_K']:.0f} K), entered from the warm-up state",
                   "precision": "fp32-mixed (FP64-exact thermal transform and FP64 reductions)"
                   if args.precision == "fp32" else "fp64",
                   "spins": lat.n, "nnz": lat.nnz, "timed_window": win32,
                   "exec": EXEC_NAMES[info32["exec"]] if info32["exec"] else "auto (captured graphs of step launches)",
                   "block": info32["block"], "tile": info32["tile"], "draw_ahead_eighths": info32["draw_ahead"],
                   "gaussian_pass": info32.get("gaussian_pass", 0), "row_patterns": info32.get("row_patterns", 0),
                   "launch_shape": "spin_system_autotune" if args.autotune_film else "library default",
                   "l2": "state 0.8 GB >> 126 MB L2, no flush needed", "replicas": world},
        "roofline": {"bound": "hbm", "achieved": kernel_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": kernel_gbs / hbm_peak,
                     "traffic": KERNEL_DRAM_BYTES[dom] if (default_shape and args.precision == "fp32") else None,
                     "traffic_source": "one ncu capture (profiles/), not measured in this run",
                     "kernel": dom, "kernel_ms": dom_ms,
                     "per_unit": f"{pass_b:.1f} B per spin per Heun pass (the two-pass byte model: S, S' and Q "
                                 f"streamed, the CSR row as stored), {lat.n} spins per launch",
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                     "step_achieved": step_gbs, "step_frac": step_gbs / hbm_peak,
                     "step_per_unit": f"{step_b:.1f} B per spin-step",
                     "layout_bytes_per_spin_step": lay_b,
                     "layout_frac": lay_b * lat.n / (ms32 / args.steps * 1e-3) / 1e9 / hbm_peak},
        "kernels_ms": kt32, "clocks": clk32,
        "e2e": {"value": world * lat.n / e2e32, "unit": "spin-steps/s", "h2d_bytes_per_step": 8,
                "d2h_bytes_per_step": 64},
        # step kernels launched in the timed region: a predictor and a corrector per step (and a
        # Gaussian pass with the split step), or one cooperative launch per 64 steps persistent
        "gpu_launches": (-(-args.steps // 64)) if info32["exec"] == 3 else
                        (3 if info32.get("gaussian_pass", 0) else 2) * args.steps,
        "final_m": [float(x) for x in mag32],
    }
    # the FP64, batched, workload, Monte Carlo, demagnetising, alternative-integrator, long-row and
    # CPU-baseline legs are single-GPU diagnostics: at N > 1 the line carries the headline only
    if not args.no_extras and world == 1:
        k64 = max(20, args.steps // 4)
        ms64, kt64, _, clk64, _, _, win64 = timed_run("fp64", k64, args.warmup, 5)
        fp64_peak = SMS * FP64_SLOTS_PER_SM_CYCLE * 2 * sm_ghz / 1e3  # TFLOP/s (FMA-slot flops)
        fp64_ach = 2 * FP64_FORM_PREDICTOR_FP64_PER_SPIN * lat.n / (kt64["predictor_ms"] * 1e-3) / 1e12
        out["fp64"] = {"value": world * lat.n * k64 / (ms64 * 1e-3), "unit": "spin-steps/s", "steps": k64,
                       "kernels_ms": kt64, "clocks": clk64,
                       "hbm_frac": step_bytes_per_spin(8, nnz_per) * lat.n / (ms64 / k64 * 1e-3) / 1e9 / hbm_peak,
                       "fp64_pipe": {"bound": "alu", "kernel": "k_predictor", "achieved": fp64_ach,
                                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": fp64_ach / fp64_peak,
                                     "per_unit": f"{FP64_FORM_PREDICTOR_FP64_PER_SPIN:.0f} FP64 instructions per "
                                                 "spin (ncu, profiles/), 2 flop-equivalents each",
                                     "peak_source": f"152 SMs x 2 FP64 slots/cycle x 2 x {sm_ghz:.3f} GHz "
                                                    "(measured clock)"}}
        out["fp32_vs_fp64"] = out["value"] / out["fp64"]["value"]  # FP32-mixed speed-up on the same GPU
        out["fp32_error"] = fp32_error(stream)
        from paper_1310_6143_gb300.system import debug_fp64_rate
        out["fp64_rate_probe"] = {f"{name}_inst_per_sm_cycle": debug_fp64_rate(m) / SMS / (sm_ghz * 1e9)
                                  for m, name in ((0, "dfma_shared_operands"), (1, "dfma_distinct_operands"),
                                                  (2, "dadd"))}
        # the batched form: 256 independent columnar grains (2,000-40,000 spins each, T
        # uniform in 0-800 K) in one handle, launch shape chosen by the autotuner
        grains, temps = L.grain_ensemble(count=256, seed=12345)
        ng = sum(g.n for g in grains)
        nnz_g = sum(g.nnz for g in grains)
        kb = max(50, args.steps // 2)

        def batch_ms(b, steps):
            b.step(args.warmup)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            e1.synchronize()
            b.sync()
            return e0.elapsed_time(e1) / steps

        with SpinSystem(grains, alpha=0.1, dt=1e-16, T=list(temps), seed=[4000 + k for k in range(256)],
                        sys_id=list(range(256)), precision="fp32", stream=stream) as b:
            tuned = b.info() if args.no_autotune else b.autotune(10)
            msb = batch_ms(b, kb)
            # the two launch forms side by side in the tuned shape: per-step captured graphs, and
            # one persistent cooperative launch per 64 steps (captured)
            forms = {}
            for mode in ("graph", "persistent"):
                b.set_exec(mode)
                forms[f"{mode}_ms"] = batch_ms(b, kb)
        gb = step_bytes_per_spin(4, nnz_g / ng)
        out["batched"] = {"value": world * ng / (msb * 1e-3), "unit": "spin-steps/s", "steps": kb,
                          "systems": 256, "spins": ng, "ms_per_step": msb,
                          "exec": EXEC_NAMES[tuned["exec"]], "block": tuned["block"], "tile": tuned["tile"],
                          "gaussian_pass": tuned.get("gaussian_pass", 0), "row_patterns": tuned.get("row_patterns", 0),
                          **forms,
                          "hbm_frac": gb * ng / (msb * 1e-3) / 1e9 / hbm_peak,
                          "hbm_per_unit": f"{gb:.1f} B per spin-step (two-pass model, mean row {nnz_g / ng:.3f})"}
        out["workloads"] = workload_table(stream, rank)
        out["mc"] = mc_table(stream, rank)
        out["demag"] = demag_table(stream, rank)
        out["midpoint"] = midpoint_table(stream, rank)
        out["long_range"] = long_range_table(stream, rank, hbm_peak=hbm_peak)
        out["cpu_baseline"] = cpu_baseline(lat, T)
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()

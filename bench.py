#!/usr/bin/env python
"""Throughput of the direct-QPAT acoustic hot path on GB300.

Workload (seeded, synthetic): 2D 512 x 512 interior at dx = 0.05 mm with a
32-cell PML on every side (576 x 576 FFT grid), six elliptic inclusions
(c 1400-1650 m/s, rho 900-1100 kg/m^3, alpha0 0.5-1.0 dB MHz^-y cm^-1),
y = 1.5, CFL 0.3, Nt = 2000, 256 sensors on the interior perimeter.  One
step = one forward H_a and one adjoint H_a^* propagation of Nt time steps
for each of ``--batch`` independent problems (initial pressures / adjoint
sources), in FP32 with FP64-built operator tables.

metric: forward+adjoint cell-steps per second, a cell-step being one FFT-grid
cell (PML included) advanced one time step by one propagation.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload instead (see ``oracle/``).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import phantoms  # noqa: E402

METRIC = "fwd+adjoint cell-steps/s"
UNIT = "cell-steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=12, help="independent problems per step")
    p.add_argument("--nt", type=int, default=None, help="override Nt (default: workload's 2000)")
    p.add_argument("--no-extras", action="store_true", help="skip fp64/e2e/roofline/cpu legs")
    p.add_argument("--n3", type=int, default=None, help="c5 only: interior nodes per axis (default 256)")
    p.add_argument("--medium-grid", default="c1", choices=["c1", "c2"],
                   help="medium workload: the 168^2 grid with 600 steps (c1) or the 576^2 grid with 2000 (c2)")
    p.add_argument("--medium-precision", default="fp64", choices=["fp64", "fp32"],
                   help="sweep precision of --workload medium (gradient sums FP64 in both)")
    p.add_argument("--ld-method", default="ld", choices=["ld", "pdipm", "admm"],
                   help="ld workload: lagged diffusivity (Algorithm 5), primal-dual interior point (Algorithm 6) "
                        "or the ADMM + L-BFGS benchmark (Algorithms 1-3)")
    p.add_argument("--workload", default="c2", choices=["c2", "c4", "c5", "ld", "medium"],
                   help="c2: the 576^2 forward+adjoint workload (default); c4: 48 Jacobian-vector "
                        "products over 288^2/432^2/576^2 grids in one graph; c5: the 3D 256^3 workload; "
                        "ld: the inexact-Newton LD reconstruction; medium: the gradient in sound speed and "
                        "density, FP64, 168^2 grid (diagnostic lines)")
    return p.parse_args()


def workload():
    return phantoms.C2


def config_dict(w, batch, nt, extra=None):
    d = {"workload": f"2d {w.n}x{w.n} interior, {w.grid}x{w.grid} FFT grid (pml {w.pml}), "
                     f"Nt={nt}, {w.n_sensors} perimeter sensors, y={w.y}, fwd+adj per problem",
         "grid": w.grid, "interior": w.n, "nt": nt, "batch": batch, "sensors": w.n_sensors,
         "seq_len": nt, "global_batch": batch,
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def _cells(w):
    return w.grid ** w.dim


def _oracle_run(w, nt_sample, seed, adjoint=True):
    """Set up the oracle for w, then return a closure that runs forward (and
    adjoint) propagations of nt_sample steps."""
    from oracle import acoustic
    S = acoustic.setup_from_workload(w, nt=nt_sample)
    p0 = phantoms.smooth_p0(w, seed)
    W = phantoms.random_field((nt_sample, w.n_sensors), seed + 1)

    def go():
        acoustic.forward(S, p0)
        if adjoint:
            acoustic.adjoint(S, W)
    return go


def oracle_rate(w, nt_sample, seed=0, adjoint=True):
    """Cell-steps/s of the FP64 oracle (forward, and adjoint unless told
    otherwise, nt_sample steps each) on this host, setup excluded."""
    go = _oracle_run(w, nt_sample, seed, adjoint)
    t0 = time.perf_counter()
    go()
    t = time.perf_counter() - t0
    return _cells(w) * nt_sample * (2 if adjoint else 1) / t, t


def _oracle_worker(w, nt_sample, seed, barrier, out, adjoint=True):
    """One oracle problem in its own (spawned) process: setup, wait for the
    other workers, then time forward (+ adjoint) of nt_sample steps."""
    go = _oracle_run(w, nt_sample, seed, adjoint)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    go()
    out.put((seed, t0, time.perf_counter()))


def host_cpu():
    """Architecture, CPU model and core count of the host running the oracle."""
    import platform
    model = platform.processor() or ""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            hit = [ln.split(":", 1)[1].strip() for ln in info if ln.split(":", 1)[0].strip() == key]
            if hit:
                model = hit[0] if key != "CPU part" else f"CPU part {hit[0]}"
                break
    except OSError:
        pass
    return {"machine": platform.machine(), "cpu": model, "nproc": os.cpu_count()}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate_parallel(w, nt_sample, procs, seed=0, adjoint=True):
    """Cell-steps/s of `procs` independent oracle problems run at once, one
    single-threaded process per core (spawned, so safe after CUDA is up).
    Timed from the common start (a barrier after setup) to the last finish."""
    import multiprocessing as mp
    import queue as _queue
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    ps = []
    try:
        ps = [ctx.Process(target=_oracle_worker, args=(w, nt_sample, seed + 2 * i, barrier, out, adjoint),
                          daemon=True)
              for i in range(procs)]
        for p in ps:
            p.start()
        res, deadline = [], time.monotonic() + 1800
        while len(res) < procs:
            try:
                res.append(out.get(timeout=2))
            except _queue.Empty:
                bad = [p.exitcode for p in ps if p.exitcode not in (None, 0)]
                if bad or time.monotonic() > deadline:
                    raise RuntimeError(f"oracle worker failed (exit codes {bad})")
        for p in ps:
            p.join(timeout=60)
    finally:
        for p in ps:
            if p.is_alive():
                p.terminate()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t = max(r[2] for r in res) - min(r[1] for r in res)
    return procs * _cells(w) * nt_sample * (2 if adjoint else 1) / t, t


def sample_nt(w, target_s, cap, adjoint=True):
    probe_nt = 6
    _, t = oracle_rate(w, probe_nt, adjoint=adjoint)
    return max(4, min(cap, int(probe_nt * target_s / max(t, 1e-3))))


def cpu_baseline(w, target_s=10.0, nt_fixed=None, adjoint=True, max_procs=None):
    """The FP64 oracle on this host: one problem per core on every core (or
    max_procs), plus the single-threaded rate for reference."""
    nt_s = nt_fixed or sample_nt(w, target_s, 400, adjoint)
    what = "forward+adjoint" if adjoint else "forward"
    v1, t1 = oracle_rate(w, nt_s, seed=1, adjoint=adjoint)
    single = {"value": v1, "cores": 1,
              "sample": f"1 problem, {what} of {nt_s} steps each ({t1:.1f} s wall)"}
    P = host_cores() if max_procs is None else min(host_cores(), max_procs)
    grid = "x".join([str(w.grid)] * w.dim)
    try:
        vp, tp = oracle_rate_parallel(w, nt_s, P, seed=11, adjoint=adjoint)
    except Exception as e:  # noqa: BLE001 - the single-thread figure still stands
        return {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"FP64 numpy oracle, 1 problem, {what} of {nt_s} steps on the {grid} grid "
                          f"({t1:.1f} s wall), single thread (the all-core run failed: {e})"}
    return {"value": vp, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": f"FP64 numpy oracle, {P} independent problems at once, one single-threaded process "
                      f"per core, {what} of {nt_s} steps each on the {grid} grid "
                      f"({tp:.1f} s wall from the common start to the last finish)",
            "single_thread": single, "host": host_cpu()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    nt = args.nt or w.nt
    for _ in range(args.warmup):
        oracle_rate(w, 4)
    nt_s = sample_nt(w, 8.0, 200)
    P = host_cores()
    cells, times, mode = 0, [], f"{P} problems at once, one single-threaded process per core"
    parallel = True
    for k in range(args.steps):
        if parallel:
            try:
                _, t = oracle_rate_parallel(w, nt_s, P, seed=100 * k)
                cells += P * w.grid * w.grid * nt_s * 2
                times.append(t)
                continue
            except Exception as e:  # noqa: BLE001 - fall back to one core, and say so
                parallel, P, mode = False, 1, f"1 problem, single thread (the all-core run failed: {e})"
        _, t = oracle_rate(w, nt_s, seed=k)
        cells += w.grid * w.grid * nt_s * 2
        times.append(t)
    value = cells / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, args.batch, nt, {"reference_sample_nt": nt_s,
                                                                  "reference_problems_per_step": P}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle", "host": host_cpu(),
                             "sample": f"each step: forward+adjoint of {nt_s} of the {nt} time steps, "
                                       f"FP64 numpy, {mode}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, path, index):
        self.path, self.index, self.proc = path, index, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_hbm_peak(fallback=6800.0):
    """HBM copy bandwidth [GB/s] measured on this machine (MEASURED_PEAKS.json),
    else the fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return fallback


def source_hash(files=None):
    """Hash of the library sources (all of csrc/, or the named files)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1810_11685_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if files is None or f in files:
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# the sources the 2D FP32 pass kernels of the bench workload are built from
PASS_SOURCES = ("fast_576.cu", "fast_kernels.cuh", "fft_reg.cuh", "fft_smem.cuh", "pass_ops.cuh",
                "qpat_internal.h", "propagate.cu")
ALL_PHASES = ["F_R1", "F_C1", "F_R2", "F_C2", "F_R3", "F_C3", "A_R1", "A_C2", "A_R3", "A_C4", "A_R5", "A_C6"]


def pass_hash():
    return source_hash(PASS_SOURCES)


def b_alg(dim, prec="f32", alpha_varies=True):
    """Algorithmic bytes per cell-step: read + write of the state z_n ((2 d + 1)
    fields) and one read of each per-cell medium coefficient (c, rho-bar,
    rho-bar_1..d, and alpha0 where it varies); tau and eta follow from c,
    alpha0 and y, and the PML, k-space tables and sensors are lower order."""
    elt = 4 if prec == "f32" else 8
    return (2 * (2 * dim + 1) + (2 + dim) + (1 if alpha_varies else 0)) * elt


def pass_bytes(phase, w, batch, elt=4):
    """Implementation bytes of one launch of a propagation pass: every input
    and output field of each problem read or written once (half spectra as
    complex values, per-problem state fields), plus the medium diagonals and
    k-space tables, which all problems of the batch share, read once."""
    G = w.grid * w.grid
    H = w.grid * (w.grid // 2 + 1)
    spec = {"F_R1": (2, 1), "F_R2": (2, 2), "F_R3": (2, 2), "A_R1": (1, 2), "A_R3": (2, 2), "A_R5": (2, 2),
            "F_C1": (1, 2), "F_C2": (2, 2), "F_C3": (2, 2), "A_C2": (2, 2), "A_C4": (2, 2), "A_C6": (2, 1)}
    state = {"F_R1": 3, "F_R2": 4, "F_R3": 4, "A_R1": 1, "A_R3": 5, "A_R5": 4}      # per problem
    medium = {"F_R1": 3, "F_R2": 2, "F_R3": 1, "A_R1": 3, "A_R3": 1, "A_R5": 2}     # shared
    tables = {"F_C1": 1, "F_C2": 1, "F_C3": 2, "A_C2": 2, "A_C4": 1, "A_C6": 1}     # shared, half grid
    kin, kout = spec[phase]
    b = batch * (kin + kout) * H * 2 * elt
    if phase in state:
        b += (batch * state[phase] + medium[phase]) * G * elt
    else:
        b += tables[phase] * H * elt
    return b


def step_traffic(batch):
    """DRAM bytes of one time step (forward or adjoint) of the batch on the
    576^2 grid, from the committed ncu capture of every pass kind, while its
    pass-source hash and batch match the present build (else None)."""
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except Exception:
        return None
    per = tr.get("per_launch", {})
    if tr.get("pass_hash") != pass_hash() or tr.get("batch") != batch or not all(p in per for p in ALL_PHASES):
        return None
    return sum(per[p] for p in ALL_PHASES) / 2.0


def roofline_step(value, dim, nt_unit_cells, prec="f32", alpha_varies=True, traffic=None, what=""):
    """Step-level roofline: the algorithmic bytes (b_alg per cell-step) of one
    time step of all problems (nt_unit_cells cell-steps) over its measured
    duration, against the measured HBM copy bandwidth."""
    B = b_alg(dim, prec, alpha_varies)
    peak = measured_hbm_peak()
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if measured_hbm_peak(fallback=None) else "fallback"
    ach = value * B / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic, "kernel": what, "b_alg_bytes_per_cell_step": B,
            "cell_steps_per_launch": nt_unit_cells,
            "alg_bytes_per_launch": B * nt_unit_cells, "peak_source": peak_src}


def timed_steps(step, steps, warmup, flush, local, dist=None, rank=0):
    """`warmup` untimed steps, then `steps` steps each bracketed by CUDA events
    on the current stream, an L2 flush between them, a barrier and a device
    synchronise on both sides, clocks sampled during the timed region.
    Returns (per-step ms, clock summary)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clk_path = os.path.join(tempfile.gettempdir(), f"qpat_clocks_{rank}.csv")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(clk_path, local) as clk:
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record()
            step()
            evs[k][1].record()
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return [a.elapsed_time(b) for a, b in evs], clk.summary()


def timed_e2e(step_host, reps, flush):
    """Mean ms of `reps` end-to-end steps (host copies inside), CUDA events."""
    import torch
    ms = []
    for k in range(reps):
        flush.fill_(float(k))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        step_host()
        e.record()
        torch.cuda.synchronize()
        ms.append(s.elapsed_time(e))
    return statistics.mean(ms)


def cufft_comparison(B, n, ms_per_time_step, lossless=False):
    """Comparison only (never on the product path): the library (cuFFT, via
    torch.fft) real 2D transforms that one time step of the batch needs --
    5 forward and 6 inverse with absorption (3 and 4 lossless) -- timed alone,
    against the measured fused step (FFTs, k-space symbols and pointwise
    updates together)."""
    import torch
    nf, ni = (3, 4) if lossless else (5, 6)
    x = torch.randn(B, n, n, device="cuda")
    X = torch.fft.rfft2(x)
    for _ in range(3):
        torch.fft.rfft2(x)
        torch.fft.irfft2(X, s=(n, n))
    torch.cuda.synchronize()
    reps = 20
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        for _ in range(nf):
            torch.fft.rfft2(x)
        for _ in range(ni):
            torch.fft.irfft2(X, s=(n, n))
    e.record()
    torch.cuda.synchronize()
    lib = s.elapsed_time(e) / reps
    return {"what": f"{nf} R2C + {ni} C2R 2D transforms of [{B}][{n}][{n}] FP32 per time step (torch.fft), "
                    f"transforms only, no k-space symbols or pointwise updates",
            "cufft_ms_per_time_step": lib, "fused_ms_per_time_step": ms_per_time_step,
            "fused_over_cufft_transforms": ms_per_time_step / lib}


def run_ours(args):
    import torch
    from paper_1810_11685_gb300.binding import context_from_workload

    from paper_1810_11685_gb300 import replicas
    rank, world, local = replicas.world()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    nt = args.nt or w.nt
    B = args.batch
    ctx = context_from_workload(w, precision="fp32", max_batch=B, nt=nt)
    G = w.grid * w.grid
    cells_per_step = B * G * nt * 2

    rng = np.random.default_rng(100 + rank)
    p0_h = np.stack([phantoms.smooth_p0(w, seed=rank * B + b) for b in range(B)]).astype(np.float32)
    w_h = rng.standard_normal((B, nt, w.n_sensors)).astype(np.float32)
    p0 = torch.as_tensor(p0_h, device=dev)
    W = torch.as_tensor(w_h, device=dev)
    data = torch.empty(B, nt, w.n_sensors, device=dev)
    padj = torch.empty(B, w.n, w.n, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.acoustic_forward(p0, out=data)
        ctx.acoustic_adjoint(W, out=padj)

    for _ in range(max(3, args.warmup)):
        step()
    ctx.sync()
    launches0 = ctx.stats()["launches"]
    ms, clocks = timed_steps(step, args.steps, 0, flush, local, dist, rank)
    ctx.sync()
    launches = ctx.stats()["launches"] - launches0
    t_ms = replicas.max_over_ranks(sum(ms), device=dev)
    value = replicas.throughput(cells_per_step * args.steps, world, t_ms / 1e3)

    extras = {}
    if not args.no_extras and rank == 0:
        # end to end through the C ABI with host buffers: pinned H2D of this
        # step's inputs, the propagations, D2H of both results
        p0_pin = torch.from_numpy(p0_h).pin_memory()
        w_pin = torch.from_numpy(w_h).pin_memory()
        out_pin = torch.empty(B, nt, w.n_sensors).pin_memory()
        adj_pin = torch.empty(B, w.n, w.n).pin_memory()

        def step_host():
            p0.copy_(p0_pin, non_blocking=True)
            W.copy_(w_pin, non_blocking=True)
            step()
            out_pin.copy_(data, non_blocking=True)
            adj_pin.copy_(padj, non_blocking=True)
        e2e_ms = timed_e2e(step_host, max(2, args.steps), flush)
        h2d = p0_h.nbytes + w_h.nbytes
        d2h = out_pin.numel() * 4 + adj_pin.numel() * 4
        extras["e2e"] = {"value": cells_per_step / (e2e_ms / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

        # step level (the headline): B_alg per cell-step over one time step of
        # the batch, from the device-timed steps above
        ms_ts = (t_ms / args.steps) / (2 * nt)
        traffic = step_traffic(B)
        extras["roofline"] = roofline_step(value / world, 2, B * G, traffic=traffic,
                                           what=f"one time step (forward or adjoint, 6 fused passes) of {B} "
                                                f"problems on the {w.grid}^2 grid, {ms_ts * 1e3:.1f} us")
        extras["roofline"]["traffic_bytes_per_cell_step"] = None if traffic is None else traffic / (B * G)

        # per pass (implementation bytes; CUDA events on the library's stream)
        per = {}
        for ph in ALL_PHASES:
            ctx.profile(ph)
            step()
            pms, n = ctx.profile_read()
            ctx.profile(None)
            per[ph] = {"ms_total": pms, "launches": n, "us_per_launch": 1e3 * pms / max(n, 1)}
        top = max(per, key=lambda k: per[k]["ms_total"])
        peak = measured_hbm_peak()
        alg = pass_bytes(top, w, B)
        ach = alg / (per[top]["us_per_launch"] * 1e-6) / 1e9
        ptraffic = None
        try:
            tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
            if tr.get("pass_hash") == pass_hash() and tr.get("batch") == B and top in tr.get("per_launch", {}):
                ptraffic = tr["per_launch"][top]
        except Exception:
            pass
        extras["roofline_impl"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                   "frac": ach / peak, "traffic": ptraffic, "kernel": top,
                                   "impl_bytes_per_launch": alg,
                                   "note": "dominant pass alone; its bytes include the FFT intermediates "
                                           "(half spectra) the method does not strictly need, and most of "
                                           "them stay in L2 at this working set"}
        extras["passes"] = {k: round(v["us_per_launch"], 2) for k, v in per.items()}
        extras["cufft"] = cufft_comparison(B, w.grid, ms_ts)

        # the plain FP64 form on the same GPU: one problem, same workload
        ctx64 = context_from_workload(w, precision="fp64", max_batch=1, nt=nt)
        p64 = p0[:1].double().contiguous()
        W64 = W[:1].double().contiguous()

        def step64():
            ctx64.acoustic_forward(p64)
            ctx64.acoustic_adjoint(W64)
        ms64, _ = timed_steps(step64, 5, 1, flush, local)
        ctx64.sync()
        v64 = [G * nt * 2 / (m / 1e3) for m in ms64]
        extras["fp64_plain"] = {"value": statistics.mean(v64), "unit": UNIT, "batch": 1, "repeats": len(v64),
                                "min": min(v64), "max": max(v64), "stdev": statistics.stdev(v64),
                                "fp32_batched_over_fp64_plain": value / world / statistics.mean(v64)}
        ctx64.close()
        extras["cpu_baseline"] = cpu_baseline(w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(w, B, nt, {"parallelism": f"replicas x{world}, no collective"}),
                "clocks": clocks, "gpu_launches": int(launches), "impl": "ours",
                "source_hash": source_hash(), "pass_hash": pass_hash()}
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_c4(args):
    """48 Jacobian-vector products of the Newton inner-loop mix: 16 problems on
    each of the 256^2, 384^2 and 512^2 interiors (288^2, 432^2, 576^2 FFT
    grids), Nt chosen so the background wave crosses the interior 1.5 times.
    The device-timed value is the acoustic half (qpat_group_propagate: the
    dominant part, one graph launch); e2e is the whole J v through
    qpat_group_jvp (diffusion solves included) from host buffers."""
    import torch
    from paper_1810_11685_gb300.binding import Group, context_from_workload
    ws = phantoms.c4_workloads()
    ctxs, p0s, cells, unit_cells = [], [], 0, 0
    for w in ws:
        c, _, _ = phantoms.acoustic_medium(w)
        nt = args.nt or phantoms.c4_nt(w, c)
        ctx = context_from_workload(w, precision="fp32", max_batch=16, nt=nt)
        ctxs.append(ctx)
        p0s.append(torch.as_tensor(phantoms.random_field((16,) + w.interior_shape, 7), dtype=torch.float32,
                                   device="cuda"))
        cells += 16 * w.grid * w.grid * nt
        unit_cells += 16 * w.grid * w.grid
    g = Group(ctxs)
    best, cands = g.tune([16, 16, 16], steps=24)
    tuned = {"shape": best, "candidates_ms_fwd_adj_24_steps": [[c, round(ms, 3)] for c, ms in cands]}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    outs = [torch.empty(16, c.nt, c.ns, device="cuda") for c in ctxs]

    def step():
        g.acoustic_forward(p0s, outs=outs)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    l0 = ctxs[0].stats()["launches"]
    ms, clocks = timed_steps(step, args.steps, 0, flush, torch.cuda.current_device())
    launches = ctxs[0].stats()["launches"] - l0
    t_ms = sum(ms)
    value = cells * args.steps / (t_ms / 1e3)
    max_nt = max(c.nt for c in ctxs)
    # e2e: qpat_group_jvp with mu and v from pinned host memory, dP back
    mus = [phantoms.optical_absorption(w) for w in ws]
    rng = np.random.default_rng(11)
    vs = []
    for w in ws:
        v = rng.standard_normal((16,) + w.interior_shape)
        vs.append(v / np.linalg.norm(v.reshape(16, -1), axis=1).reshape((16,) + (1,) * w.dim))
    mu_pin = [torch.from_numpy(np.ascontiguousarray(m)).pin_memory() for m in mus]
    v_pin = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in vs]
    mu_d = [torch.empty(m.shape, dtype=torch.float64, device="cuda") for m in mu_pin]
    v_d = [torch.empty(v.shape, dtype=torch.float64, device="cuda") for v in v_pin]
    dP_pin = [torch.empty(16, c.nt, c.ns).pin_memory() for c in ctxs]

    def step_host():
        for a, b in zip(mu_d + v_d, mu_pin + v_pin):
            a.copy_(b, non_blocking=True)
        dP = g.jvp(mu_d, v_d, 0b0001)
        for a, b in zip(dP_pin, dP):
            a.copy_(b, non_blocking=True)
    step_host()
    torch.cuda.synchronize()
    e2e_ms = timed_e2e(step_host, max(2, args.steps), flush)
    h2d = sum(t.numel() * 8 for t in mu_pin + v_pin)
    d2h = sum(t.numel() * 4 for t in dP_pin)
    ms_ts = (t_ms / args.steps) / max_nt
    line = {"metric": "jvp cell-steps/s (acoustic half of 48 J v over 3 grids, one launch per pass kind)"
                      if best["multi"] else "jvp cell-steps/s (acoustic half of 48 J v over 3 grids, one graph)",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": "c4: 16 x 288^2 + 16 x 432^2 + 16 x 576^2 FFT grids (256^2/384^2/512^2 "
                                   "interiors), acoustic forward of J v per problem, Nt crossing 1.5 interiors",
                       "nt": [c.nt for c in ctxs], "batch_per_grid": 16,
                       "l2": "flushed between timed steps (256 MiB write); working set above L2"},
            "clocks": clocks, "gpu_launches": int(launches), "autotuned": tuned,
            "roofline": roofline_step(value, 2, unit_cells,
                                      what=f"one time step of all 48 problems while all three grids step "
                                           f"(mean {ms_ts * 1e3:.1f} us over the {max_nt}-step call)"),
            "e2e": {"value": cells / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "what": "qpat_group_jvp: 48 diffusion solves and jvp heatings, then the acoustic forwards, "
                            "from pinned host mu and v, dP back to the host"}}
    if not args.no_extras:
        rates = []
        for w, c in zip(ws, ctxs):
            rates.append(cpu_baseline(dataclasses.replace(w, nt=c.nt), target_s=6.0, adjoint=False))
        tot_cells = sum(16 * w.grid * w.grid * c.nt for w, c in zip(ws, ctxs))
        tot_time = sum(16 * w.grid * w.grid * c.nt / r["value"] for w, c, r in zip(ws, ctxs, rates))
        line["cpu_baseline"] = {"value": tot_cells / tot_time, "unit": UNIT, "cores": rates[0]["cores"],
                                "kind": "oracle",
                                "sample": "the three grids' rates, weighted by their share of the cell-steps; "
                                          + " | ".join(r["sample"] for r in rates),
                                "per_grid": [r["value"] for r in rates]}
    print(json.dumps(line), flush=True)


def run_c5(args):
    """3D workload: 256^3 interior, 16-cell PML (288^3 FFT grid), 128 x 128
    planar sensors, forward + adjoint of one problem in FP32, Nt = 1500."""
    import torch
    from paper_1810_11685_gb300.binding import context_from_workload
    w = phantoms.C5 if not args.n3 else dataclasses.replace(phantoms.C5, n=args.n3)
    nt = args.nt or w.nt
    ctx = context_from_workload(w, precision="fp32", max_batch=1, nt=nt)
    p0_h = phantoms.smooth_p0(w).astype(np.float32)[None]
    w_h = np.random.default_rng(5).standard_normal((1, nt, w.n_sensors)).astype(np.float32)
    p0 = torch.as_tensor(p0_h, device="cuda")
    W = torch.as_tensor(w_h, device="cuda")
    data = torch.empty(1, nt, w.n_sensors, device="cuda")
    padj = torch.empty((1,) + w.interior_shape, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        ctx.acoustic_forward(p0, out=data)
        ctx.acoustic_adjoint(W, out=padj)
    for _ in range(max(3, args.warmup)):
        step()
    ctx.sync()
    l0 = ctx.stats()["launches"]
    ms, clocks = timed_steps(step, args.steps, 0, flush, torch.cuda.current_device())
    ctx.sync()
    launches = ctx.stats()["launches"] - l0
    t_ms = sum(ms)
    G = w.grid ** 3
    cells = G * nt * 2
    value = cells * args.steps / (t_ms / 1e3)
    p0_pin = torch.from_numpy(p0_h).pin_memory()
    w_pin = torch.from_numpy(w_h).pin_memory()
    out_pin = torch.empty(data.shape).pin_memory()
    adj_pin = torch.empty(padj.shape).pin_memory()

    def step_host():
        p0.copy_(p0_pin, non_blocking=True)
        W.copy_(w_pin, non_blocking=True)
        step()
        out_pin.copy_(data, non_blocking=True)
        adj_pin.copy_(padj, non_blocking=True)
    e2e_ms = timed_e2e(step_host, max(2, args.steps), flush)
    ms_ts = (t_ms / args.steps) / (2 * nt)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": f"c5: 3D {w.n}^3 interior, {w.grid}^3 FFT grid (pml {w.pml}), "
                                   f"{w.n_sensors} planar sensors, y={w.y}, fwd+adj, Nt={nt}", "nt": nt,
                       "batch": 1, "l2": "flushed between timed steps (256 MiB write); working set above L2"},
            "clocks": clocks, "gpu_launches": int(launches),
            "roofline": roofline_step(value, 3, G, alpha_varies=False,
                                      what=f"one time step (forward or adjoint, 12 fused passes) on the "
                                           f"{w.grid}^3 grid, {ms_ts * 1e3:.1f} us"),
            "e2e": {"value": cells / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(p0_h.nbytes + w_h.nbytes),
                    "d2h_bytes_per_step": int(out_pin.numel() * 4 + adj_pin.numel() * 4)}}
    if not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(w, nt_fixed=2, max_procs=8)
    print(json.dumps(line), flush=True)


def run_ld(args):
    """Simultaneous (kappa, mu) reconstruction by the inexact-Newton LD method
    (Algorithms 4 and 5, qpat_ld_solve) on the 128^2 interior of the 2D
    circle-sensor workload (168^2 FFT grid, 600 samples, 128 sensors), four
    illuminated sides, FP32 propagation: synthetic data from a seeded mu with
    three discs and a seeded log-normal kappa (30 % spread about the
    workload's value), initial guesses the background values."""
    import torch
    from paper_1810_11685_gb300.binding import context_from_workload
    w = phantoms.C1
    nt = args.nt or w.nt
    ctx = context_from_workload(w, precision="fp32", nt=nt, max_batch=4)
    rng = np.random.default_rng(w.seed + 77)
    kappa_bg = phantoms.optical_diffusion(w)
    kappa_true = torch.as_tensor(kappa_bg * np.exp(0.3 * rng.standard_normal(w.interior_shape)), device="cuda")
    mu_true = torch.as_tensor(phantoms.optical_absorption(w), device="cuda")
    illums = (1, 2, 4, 8)
    ctx.set_kappa(kappa_true)
    data = torch.stack([ctx.forward(mu_true, q)[0] for q in illums])
    mu0 = torch.full(w.interior_shape, w.mu_bg, dtype=torch.float64, device="cuda")
    kappa0 = torch.as_tensor(kappa_bg, device="cuda")
    kw = dict(k_max=3, i_max=4, i_m=4, tol_in=0.0, tol_out=0.0)
    if args.ld_method == "pdipm":
        kw.update(method="pdipm", i_max=2, i_m=2, kp_max=2, tol_med=-1.0, beta=1e-6)
    elif args.ld_method == "admm":
        kw = dict(method="admm", k_max=3, j_max=4, tol_out=0.0, lower=0.05, upper=20.0)
    ctx.ld_solve(data, illums, mu0, kappa0, k_max=1, i_max=2)      # warm-up (graphs, multigrid)
    torch.cuda.synchronize()
    times, res = [], None
    for _ in range(max(1, args.steps)):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        res = ctx.ld_solve(data, illums, mu0, kappa0, **kw)
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e) / 1e3)
    (kappa, mu), eps, inner, info = res
    t = statistics.median(times)
    G = w.grid * w.grid
    cells = info["products"] * G * nt

    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    line = {"metric": "LD reconstruction: propagation cell-steps/s inside qpat_ld_solve", "value": cells / t,
            "unit": UNIT, "n_gpus": 1, "steps": len(times), "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": f"2d {w.n}x{w.n} interior, {w.grid}x{w.grid} FFT grid, Nt={nt}, "
                                   f"{w.n_sensors} sensors, 4 illuminations, joint (kappa, mu), "
                                   + {"ld": "LD, k_max=3, i_max=i_m=4",
                                      "pdipm": "PD-IPM, k_max=3, k'_max=2, i_max=i_m=2",
                                      "admm": "ADMM + L-BFGS, k_max=3, j_max=4"}[args.ld_method], "nt": nt,
                       "method": args.ld_method},
            "seconds_per_solve": t, "outer": info["outer"], "inner": inner, "products": info["products"],
            "tv_cg_iterations": info["tv_iters"], "seconds_per_outer": t / max(1, info["outer"]),
            "seconds_by_phase": info["seconds"],
            "eps": eps,
            "rel_error": {"mu_initial": rel(mu0, mu_true), "mu_final": rel(mu, mu_true),
                          "kappa_initial": rel(kappa0, kappa_true), "kappa_final": rel(kappa, kappa_true)}}
    print(json.dumps(line), flush=True)


def run_medium(args):
    """Gradient of <w, H_a p0> in the sound speed and the density
    (qpat_vjp_medium) and the tangent J_c dc + J_rho drho (qpat_jvp_medium),
    with FP64 sweeps (or FP32 sweeps and FP64 gradient sums with
    --medium-precision fp32), on the 128^2 interior of the 2D circle-sensor workload (168^2 FFT
    grid, 600 samples, 128 sensors), or with --medium-grid c2 on the 512^2
    bench workload (576^2 grid, 2000 samples, 256 sensors).  A cell-step is one FFT-grid cell
    advanced one time step by one sweep: the gradient runs the forward sweep
    (keeping its history) and the reverse sweep, the tangent one paired sweep."""
    import torch
    from paper_1810_11685_gb300.binding import context_from_workload
    w = phantoms.C1 if args.medium_grid == "c1" else phantoms.C2
    nt = args.nt or w.nt
    prec = args.medium_precision
    ctx = context_from_workload(w, precision=prec, nt=nt)
    c, rho, _ = phantoms.acoustic_medium(w)
    rng = np.random.default_rng(w.seed + 5)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    p0 = dev(phantoms.smooth_p0(w, 2))
    dc = dev(c * 0.05 * rng.standard_normal(c.shape))
    drho = dev(rho * 0.05 * rng.standard_normal(rho.shape))
    W = dev(rng.standard_normal((nt, w.n_sensors)))
    ctx.vjp_medium(p0, W)
    ctx.jvp_medium(p0, dc, drho)
    torch.cuda.synchronize()

    def timed(fn):
        ts, l0 = [], ctx.stats()["launches"]
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)      # both calls synchronise the stream
        return statistics.median(ts), (ctx.stats()["launches"] - l0) // max(1, args.steps)

    tv, lv = timed(lambda: ctx.vjp_medium(p0, W))
    tj, lj = timed(lambda: ctx.jvp_medium(p0, dc, drho))
    G = w.grid * w.grid
    # the plain forward + adjoint of the same problem and precision, for scale
    dt_ctx = torch.float64 if prec == "fp64" else torch.float32
    p0b, Wb = p0.unsqueeze(0).to(dt_ctx), W.unsqueeze(0).to(dt_ctx)
    ctx.acoustic_forward(p0b)
    ctx.acoustic_adjoint(Wb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.acoustic_forward(p0b)
    ctx.acoustic_adjoint(Wb)
    torch.cuda.synchronize()
    tfa = time.perf_counter() - t0
    line = {"metric": "medium gradient (c, rho): cell-steps/s", "value": G * nt * 2 / tv, "unit": UNIT,
            "n_gpus": 1, "steps": max(1, args.steps), "higher_is_better": True,
            "dtype": "f64" if prec == "fp64" else "f32 sweeps, f64 gradient sums",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": f"2d {w.n}x{w.n} interior, {w.grid}x{w.grid} FFT grid, Nt={nt}, "
                                   f"{w.n_sensors} sensors, y={w.y}, gradient in c and rho", "nt": nt},
            "seconds_per_gradient": tv, "launches_per_gradient": lv, "us_per_launch_gradient": 1e6 * tv / lv,
            "seconds_per_tangent": tj, "launches_per_tangent": lj, "us_per_launch_tangent": 1e6 * tj / lj,
            "tangent_cell_steps_per_s": G * nt / tj,
            f"seconds_{prec}_forward_plus_adjoint": tfa, "gradient_over_forward_plus_adjoint": tv / tfa}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "ours" and args.workload == "c4":
        run_c4(args)
        return
    if args.impl == "ours" and args.workload == "c5":
        run_c5(args)
        return
    if args.impl == "ours" and args.workload == "ld":
        run_ld(args)
        return
    if args.impl == "ours" and args.workload == "medium":
        run_medium(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

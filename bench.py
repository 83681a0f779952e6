#!/usr/bin/env python
"""Benchmark of the FFT Toeplitz apply (and the solves around it) on GB300.

Workload (one "step"): y = A u for 65 fields on the 1023 x 1023 interior grid
of (-1, 1)^2, alpha = 1.2, quadratic basis (p = 2), FP32, 2048^2 circulant
embedding: the exact solution (1-|x|^2)_+^{1+alpha/2} plus 64 seeded smooth
random fields.  Inputs (272 MB) and the intermediate spectra (545 MB) exceed
the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With N > 1 (torchrun) every rank runs the same workload
on its own GPU (replicas; no collective on the data path) and rank 0 reports
the whole-job rate.  --impl reference times the FP64 CPU oracle on the same
workload (bounded sample of rows).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Toeplitz apply GDOF/s; Poisson solves/s @1e-10 vs FP64 plain; p50/p99 latency"
D, NSIDE, ALPHA, DEGREE, NFIELDS = 2, 1023, 1.2, 2, 65
WORKLOAD = ("2D FFT-Toeplitz apply, 1023^2 interior grid on a 2048^2 circulant embedding, alpha=1.2, "
            "quadratic basis, 65 fields (exact solution + 64 seeded smooth fields), FP32")


def workload_fields() -> np.ndarray:
    u0 = synth.ball_power(D, NSIDE, 1 + ALPHA / 2)[None]
    return np.concatenate([u0, synth.smooth_fields(D, NSIDE, NFIELDS - 1)]).astype(np.float32)


def config(parallelism: str) -> dict:
    wl = WORKLOAD if NFIELDS == 65 else WORKLOAD.replace("65 fields (exact solution + 64 seeded smooth fields)",
                                                         f"{NFIELDS} fields (profiling case)")
    return {"workload": wl, "grid": [NSIDE, NSIDE], "fft": [2048, 2048], "fields": NFIELDS,
            "alpha": ALPHA, "degree": DEGREE, "global_batch": NFIELDS, "parallelism": parallelism,
            "l2": "inputs 272 MB and spectra 545 MB exceed the 129 MB L2; no flush"}


# ---------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_generator() -> tuple:
    """The oracle's generator and c_{d,alpha} for the workload, and the seconds the build took."""
    from oracle import frac_oracle as O
    N = NSIDE + 1
    t0 = time.perf_counter()
    a = O.stencil(D, N, 2.0 / N, ALPHA, DEGREE)
    return a, O.c_dalpha(D, ALPHA), time.perf_counter() - t0


def _pool_init(a, c, fields):
    global _POOL_STATE
    _POOL_STATE = (a, c, fields)


def _pool_rows(args):
    """One worker's share of the CPU baseline: oracle rows of seeded fields and points
    until `seconds` have elapsed; returns (rows, seconds)."""
    from oracle import frac_oracle as O
    seed, seconds = args
    a, c, fields = _POOL_STATE
    rng = np.random.default_rng(seed)
    rows = 0
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < seconds:
        b = rows % len(fields)
        O.apply_rows(a, c, fields[b], rng.integers(0, NSIDE, size=(1, 2)))
        rows += 1
    return rows, time.perf_counter() - t1


class OraclePool:
    """The FP64 oracle on every host core: a pool of `spawn` workers (the parent may
    already hold a CUDA context), each evaluating dense rows of the workload with
    oracle.apply_rows (a math.fsum over the 1023^2 products of one output point)."""

    def __init__(self, gen: tuple, fields: np.ndarray, workers: int | None = None):
        import multiprocessing as mp
        self.a, self.c, self.t_gen = gen
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_pool_init,
                                                 initargs=(self.a, self.c, fields))
        self.pool.map(_pool_rows, [(w, 0.05) for w in range(self.workers)])  # workers up and warm
        self.calls = 0

    def rate(self, seconds: float) -> dict:
        self.calls += 1
        t0 = time.perf_counter()
        res = self.pool.map(_pool_rows, [(1000 * self.calls + w, seconds) for w in range(self.workers)])
        wall = time.perf_counter() - t0
        rows = sum(r for r, _ in res)
        return {"value": rows / wall / 1e9, "unit": "GDOF/s", "cores": self.workers, "kind": "oracle",
                "sample": f"{rows} output points of the 1023^2 FP64 dense sum (oracle.apply_rows, math.fsum over "
                          f"1023^2 products each) on {self.workers} worker processes for {wall:.1f} s; generator "
                          f"build {self.t_gen:.1f} s excluded"}

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_rows_rate(seconds: float = 15.0) -> dict:
    fields = np.stack([synth.ball_power(D, NSIDE, 1 + ALPHA / 2), synth.smooth_field(D, NSIDE, synth.BASE_SEED)])
    pool = OraclePool(oracle_generator(), fields)
    try:
        return pool.rate(seconds)
    finally:
        pool.close()


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    fields = np.stack([synth.ball_power(D, NSIDE, 1 + ALPHA / 2), synth.smooth_field(D, NSIDE, synth.BASE_SEED)])
    pool = OraclePool(oracle_generator(), fields)
    per_step = max(0.25, min(10.0, 60.0 / max(args.steps + args.warmup, 1)))  # about a minute in all
    for _ in range(args.warmup):
        pool.rate(min(per_step, 1.0))
    t0 = time.perf_counter()
    vals = [pool.rate(per_step) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    pool.close()
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config("host cores, rank 0 only"),
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (self.out or "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def profile_read(lib) -> dict:
    import ctypes

    class KS(ctypes.Structure):
        _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]
    arr = (KS * 64)()
    cnt = ctypes.c_int()
    lib.frac_profile_read(ctypes.cast(arr, ctypes.c_void_p), 64, ctypes.byref(cnt), 1)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(cnt.value, 64))}


def algorithmic_bytes(kernel: str, fields: float, launches: float = 1.0) -> float:
    """Compulsory bytes of each apply kernel over `fields` fields processed in
    `launches` launches (FP32; n = 1023, K = 1025 half-spectrum columns, complex
    = 8 B; the symbol pass reads the K^2 FP32 symbol once per launch)."""
    n, K = NSIDE, 1025
    u = n * n * 4
    W = n * K * 8
    if kernel.startswith("rows_fwd"):
        return fields * (u + W)
    if kernel.startswith("rows_inv"):
        return fields * (W + u)
    if kernel.startswith("cols_sym"):
        return fields * 2 * W + launches * K * K * 4
    raise KeyError(kernel)


def nominal_flops(kernel: str, fields: int) -> float:
    """Nominal FFT arithmetic per launch, 5 M log2 M per complex FFT of length
    M = 2048: the row passes do ceil(n/2) line FFTs per field, the symbol pass
    a forward and an inverse FFT on each of the K columns."""
    M, K, n = 2048, 1025, NSIDE
    per = 5.0 * M * math.log2(M)
    if kernel.startswith("rows"):
        return fields * ((n + 1) // 2) * per
    if kernel.startswith("cols_sym"):
        return fields * 2 * K * per
    raise KeyError(kernel)


def apply3d_alu_view(applies: dict, alu_peaks: dict) -> dict:
    """Nominal FFT arithmetic of the 3D 255^3 apply (M = 512 on every axis, K = 257) against
    the measured FMA rates: rows ceil(n/2) n line FFTs forward and inverse, the y passes
    n K forward and inverse, the z (symbol) pass M K forward and inverse; 5 M log2 M each."""
    n, M, K = 255, 512, 257
    per = 5.0 * M * math.log2(M)
    flops = 2 * per * (((n + 1) // 2) * n + n * K + M * K)
    out = {"nominal_flops": flops}
    for dt, key in (("f32", "3d_n255_f32_ms"), ("f64", "3d_n255_f64_ms")):
        tf = flops / (applies[key] * 1e-3) / 1e12
        out[dt] = {"achieved_tflops": tf, "frac_of_measured_fma_rate": tf / alu_peaks[dt]}
    return out


def apply_model_bytes(fields: int) -> float:
    """Whole-apply byte model B_model: read u, write y, read the symbol once,
    and the half spectrum W written and read twice (rows -> columns -> rows)."""
    n, K = NSIDE, 1025
    return fields * (2 * n * n * 4 + 4 * n * K * 8) + K * K * 4


# DRAM bytes per field (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch / fields in it) of the kernels as they stand, from one ncu capture of
# the 65-field apply (profiles/apply2d_1023_65fields_ncu_full.md), scaled to a launch
# by the fields it processes.  Remove an entry when its kernel changes.
DRAM_TRAFFIC_PER_FIELD = {
    "rows_fwd_f32_M2048": (274.043136e6 + 492.188672e6) / 65,
    "cols_sym2_f32_M2048": (551.528960e6 + 484.491520e6) / 65,
    "rows_inv_f32_M2048": (546.940672e6 + 239.797760e6) / 65,
}


def max_over_ranks(x: float, dist, device: str = "cuda") -> float:
    """The largest x over the ranks (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Replicas: every rank processes units_per_rank; the job rate is all units over the
    slowest rank's time (weak scaling, no collective on the data path)."""
    return world * units_per_rank / seconds


def run_ours(args) -> None:
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2103_03658_gb300 as fg
    from paper_2103_03658_gb300 import _native as nat
    lib = nat.load()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    alu_peaks = {k: nat.alu_peak_tflops(k) for k in ("f32", "f64", "f32x2")}
    op = fg.FracOp(D, NSIDE, ALPHA, degree=DEGREE)
    host = workload_fields()
    u = torch.from_numpy(host).cuda()
    y = torch.empty_like(u)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        op.apply(u, out=y)
    barrier()
    lib.frac_profile_enable(1)
    profile_read(lib)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            op.apply(u, out=y)
        ev1.record(stream)
        barrier()
    lib.frac_profile_enable(0)
    prof = profile_read(lib)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist)
    dof = NFIELDS * NSIDE * NSIDE
    value = whole_job_rate(dof, world, ms * 1e-3) / 1e9
    launches = sum(v[0] for v in prof.values())

    # roofline of the dominant kernel (largest total device time in the timed region):
    # algorithmic bytes of one launch over its CUDA-event duration against the measured
    # HBM copy rate; its FFT arithmetic against the FP32 rate measured in this run
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_note = "measured (STREAM-style copy)" if peak else "fallback 6800 GB/s"
    peak = peak or 6800.0
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = None
    if dom:
        name, (nl, tot) = dom
        lps = nl / args.steps
        per_launch_ms = tot / nl
        ab = algorithmic_bytes(name, NFIELDS, lps) / lps
        fl = nominal_flops(name, NFIELDS) / lps
        hbm = ab / (per_launch_ms * 1e-3) / 1e9
        alu = fl / (per_launch_ms * 1e-3) / 1e12
        tr = DRAM_TRAFFIC_PER_FIELD.get(name)
        if tr is not None:
            tr = tr * NFIELDS / lps
        bm = apply_model_bytes(NFIELDS)
        total_ms = sum(v[1] for v in prof.values())
        roof = {"bound": "hbm", "kernel": name, "achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak,
                "peak_source": peak_note, "traffic": tr,
                "algorithmic_bytes": ab, "ms_per_launch": per_launch_ms, "launches_per_step": lps,
                "fields_per_launch": NFIELDS / lps, "kernel_ms_per_step": tot / args.steps,
                "apply_model": {"bytes": bm, "ms": ms, "achieved_gbs": bm / (ms * 1e-3) / 1e9,
                                "frac_of_hbm_peak": bm / (ms * 1e-3) / 1e9 / peak},
                "alu_view": {"nominal_flops": fl, "achieved_tflops": alu, "peak_tflops": alu_peaks["f32"],
                             "frac": alu / alu_peaks["f32"], "peak_source": "fma.rn.f32 rate measured in this run",
                             "peak_f32x2_tflops": alu_peaks["f32x2"]},
                "kernels": {k: {"launches": v[0], "ms_per_launch": v[1] / max(v[0], 1),
                                "share": v[1] / max(total_ms, 1e-12)} for k, v in prof.items()}}

    # end to end through the public API with pinned host buffers (copies inside the timed region)
    hu = torch.from_numpy(host).pin_memory()
    hy = torch.empty_like(hu).pin_memory()
    op.apply(hu, out=hy)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        op.apply(hu, out=hy)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    e2e = {"value": whole_job_rate(dof, world, e2e_s) / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": host.nbytes,
           "d2h_bytes_per_step": host.nbytes}

    extra = {"alu_peaks_tflops": alu_peaks, "apply_f64": apply_f64_measurement(lib, torch, u, op, barrier,
                                                                                  alu_peaks["f64"], peak)}
    if not args.no_extra:
        extra.update(extra_measurements(fg, torch, u, op, barrier))
        extra["applies"]["3d_n255_alu_view"] = apply3d_alu_view(extra["applies"], alu_peaks)

    if rank != 0:
        op.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = oracle_rows_rate(12.0)
    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config("replicas" if world > 1 else "single GPU"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "extra": extra}
    print(json.dumps(line), flush=True)
    op.close()
    if dist is not None:
        dist.destroy_process_group()


def apply_f64_measurement(lib, torch, u32, op, barrier, f64_peak: float, hbm_peak: float, steps: int = 10) -> dict:
    """The same 65-field apply in FP64 (BASELINE config 2's FP64 arm): CUDA events over
    `steps` applies after a warm-up, per-kernel times from the library's profiler, and
    the FP64 ALU roofline (nominal FFT flops against the fma.rn.f64 rate measured in
    this run: FP64 runs at a small fraction of the FP32 rate on this part, so these
    passes are bound by FP64 arithmetic, not by HBM) beside the HBM view of the byte
    model (every FP32 byte doubled)."""
    u64 = u32.double()
    y64 = torch.empty_like(u64)
    for _ in range(2):
        op.apply(u64, out=y64)
    barrier()
    lib.frac_profile_enable(1)
    profile_read(lib)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        op.apply(u64, out=y64)
    e1.record()
    barrier()
    lib.frac_profile_enable(0)
    prof = profile_read(lib)
    ms = e0.elapsed_time(e1) / steps
    fl = sum(nominal_flops(k, NFIELDS) for k in prof)
    bm = 2 * apply_model_bytes(NFIELDS)
    del u64, y64
    return {"value": NFIELDS * NSIDE * NSIDE / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms,
            "alu_roofline": {"bound": "alu", "nominal_flops": fl, "achieved_tflops": fl / (ms * 1e-3) / 1e12,
                             "peak_tflops": f64_peak, "frac": fl / (ms * 1e-3) / 1e12 / f64_peak,
                             "peak_source": "fma.rn.f64 rate measured in this run"},
            "hbm_view": {"bytes": bm, "achieved_gbs": bm / (ms * 1e-3) / 1e9,
                         "frac": bm / (ms * 1e-3) / 1e9 / hbm_peak},
            "kernels": {k: {"launches": v[0], "ms_per_launch": v[1] / max(v[0], 1)} for k, v in prof.items()}}


def extra_measurements(fg, torch, u32, op, barrier) -> dict:
    """FP64 apply of the same workload, and solves at a 1e-10 relative residual:
    1D (n = 1023, p = 1, alpha in {0.5, 1, 1.5}) mixed and plain FP64, the 3D
    solve (255^3, p = 1) mixed at alpha in {0.4, 1.6} and plain FP64 at 0.4, the
    256-problem batch and the served stream."""
    out = {}
    solves = {}
    for alpha in (0.5, 1.0, 1.5):
        op1 = fg.FracOp(1, 1023, alpha, degree=1)
        f = torch.tensor(synth.ball_power_rhs(1, 1023, alpha), device="cuda")
        res = {}
        for prec in ("mixed", "f64"):
            op1.solve(f, precision=prec)
            barrier()
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                _, info = op1.solve(f, rtol=1e-10, precision=prec)
            barrier()
            dt = (time.perf_counter() - t0) / reps
            res[prec] = {"solves_per_s": 1.0 / dt, "ms": 1e3 * dt, "iters": info["iters"],
                         "outer": info["outer"], "rel_resid": info["rel_resid"]}
        solves[f"1d_n1023_p1_alpha{alpha}"] = res
        op1.close()
    for alpha, precs in ((0.4, ("mixed", "f64")), (1.6, ("mixed",))):
        op3 = fg.FracOp(3, 255, alpha, degree=1)
        f3 = torch.tensor(synth.ball_power_rhs(3, 255, alpha), device="cuda")
        res = {}
        for prec in precs:
            op3.solve(f3, rtol=1e-10, precision=prec)  # warm-up: kernel loading, graph instantiation
            barrier()
            t0 = time.perf_counter()
            _, info = op3.solve(f3, rtol=1e-10, precision=prec)
            barrier()
            dt = time.perf_counter() - t0
            res[prec] = {"solves_per_s": 1.0 / dt, "ms": 1e3 * dt, "iters": info["iters"], "outer": info["outer"],
                         "rel_resid": info["rel_resid"]}
        solves[f"3d_n255_p1_alpha{alpha}"] = res
        op3.close()
    out["solves"] = solves
    out["applies"] = apply_measurement(fg, torch, barrier)
    out["precond"] = precond_measurement(fg, torch, barrier)
    out["operator_builds"] = build_measurement(fg, barrier)
    out["boundary"] = boundary_measurement(fg, torch, barrier)
    out["batch"] = batch_measurement(fg, torch, barrier)
    out["batch_fft_auto"] = batch_measurement(fg, torch, barrier, fft="auto")
    out["mixed_radix"] = mixed_radix_measurement(fg, torch, barrier)
    out["served"] = served_measurement(fg, torch, barrier)
    return out


def mixed_radix_measurement(fg, torch, barrier, cases=None) -> dict:
    """The same problems on power-of-two and on mixed-radix (7-smooth) FFT lengths: FP32
    and FP64 applies (CUDA events over 10 applies of a batch of fields, alpha = 1.3,
    p = 1) and a mixed-precision solve to 1e-10; the length "auto" picks is reported."""
    out = {}
    for d, n, batch in ((1, 1100, 512), (2, 300, 64), (2, 600, 64), (2, 700, 16), (3, 200, 2)):
        if cases is not None and f"{d}d_n{n}_b{batch}" not in cases:
            continue
        row = {"auto_picks": fg.fft_length(n, d, "auto")}
        for fft in ("pow2", "smooth"):
            op = fg.FracOp(d, n, 1.3, degree=1, fft=fft)
            rec = {"fft_len": op.info()["fft_lens"][0]}
            g = torch.Generator(device="cuda").manual_seed(d * 1000 + n)
            u32 = torch.randn((batch,) + (n,) * d, device="cuda", generator=g)
            for dt, key in ((torch.float32, "apply_f32_ms"), (torch.float64, "apply_f64_ms")):
                u = u32.to(dt)
                y = torch.empty_like(u)
                for _ in range(2):
                    op.apply(u, out=y)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(10):
                    op.apply(u, out=y)
                e1.record()
                barrier()
                rec[key] = e0.elapsed_time(e1) / 10
            f = u32[0].double()
            op.solve(f, rtol=1e-10)
            barrier()
            t0 = time.perf_counter()
            _, info = op.solve(f, rtol=1e-10)
            barrier()
            rec["solve_mixed_ms"] = 1e3 * (time.perf_counter() - t0)
            rec["solve_iters"] = info["iters"]
            rec["solve_rel_resid"] = info["rel_resid"]
            row[fft] = rec
            op.close()
        out[f"{d}d_n{n}_b{batch}"] = row
    return out


def apply_measurement(fg, torch, barrier) -> dict:
    """Single-vector applies of the other configurations: 1D n = 1023 (p = 1, alpha = 1.5) in
    FP64 and FP32 (microseconds per apply, a latency: one small convolution), and 3D 255^3
    (p = 1, alpha = 1.6) in FP32 and FP64 (milliseconds per apply); CUDA events over 20 applies."""
    out = {}
    for name, (d, n, p, alpha), dtypes, scale in (("1d_n1023", (1, 1023, 1, 1.5), (torch.float64, torch.float32), 1e3),
                                                  ("3d_n255", (3, 255, 1, 1.6), (torch.float32, torch.float64), 1.0)):
        op = fg.FracOp(d, n, alpha, degree=p)
        for dt in dtypes:
            u = torch.tensor(synth.ball_power(d, n, 1 + alpha / 2), dtype=dt, device="cuda")
            y = torch.empty_like(u)
            for _ in range(3):
                op.apply(u, out=y)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                op.apply(u, out=y)
            e1.record()
            barrier()
            unit = "us" if scale == 1e3 else "ms"
            out[f"{name}_{'f64' if dt == torch.float64 else 'f32'}_{unit}"] = e0.elapsed_time(e1) / 20 * scale
        op.close()
    return out


def precond_measurement(fg, torch, barrier, lib=None) -> dict:
    """The tau preconditioner (frac_precond) of the benchmark operator (2D 1023^2, alpha = 1.2,
    p = 2) on 65 seeded fields, FP32 and FP64, and of the 3D 255^3 operator (p = 1, alpha = 0.4)
    on one field: ms per call (CUDA events over 10 calls, 3 for FP64, after 3 warm-up calls) and
    the device time per call of each kernel (the library's profiler)."""
    from paper_2103_03658_gb300 import _native
    lib = lib or _native.load()
    out = {}
    for name, (d, n, p, alpha, fields) in (("2d_n1023_65fields", (2, 1023, 2, 1.2, 65)),
                                           ("3d_n255", (3, 255, 1, 0.4, 1))):
        op = fg.FracOp(d, n, alpha, degree=p)
        g = torch.Generator(device="cuda").manual_seed(d * 100 + n)
        for dt, reps in ((torch.float32, 10), (torch.float64, 3)):
            r = torch.randn((fields,) + op.shape, dtype=dt, device="cuda", generator=g)
            for _ in range(3):
                op.precond(r)
            barrier()
            lib.frac_profile_enable(1)
            profile_read(lib)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                op.precond(r)
            e1.record()
            barrier()
            lib.frac_profile_enable(0)
            prof = profile_read(lib)
            out[f"{name}_{'f64' if dt == torch.float64 else 'f32'}"] = {
                "ms": e0.elapsed_time(e1) / reps,
                "kernels_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()}}
        op.close()
    return out


def boundary_measurement(fg, torch, barrier) -> dict:
    """frac_boundary (near field of exterior data g = exp(-|x|^2), device buffers) at the largest
    grid of each dimension: ms per call (3 calls after one warm-up; the call synchronises) and the
    nominal FP64 rate of its line FFTs (5 M' log2 M' flops per line, M' = nextpow2(3N - 1), the
    lines each pass transforms, M'/2 + 1 along axis 0 after the first); d = 1 is a direct sum
    (2N + 1 products per point)."""
    out = {}
    for name, (d, n, p, alpha) in (("1d_n4095", (1, 4095, 1, 1.5)), ("2d_n1023", (2, 1023, 2, 1.2)),
                                   ("3d_n255", (3, 255, 1, 1.6))):
        op = fg.FracOp(d, n, alpha, degree=p)
        # g = exp(-|x|^2) on the extended grid, formed on the device from the axis coordinates
        x = torch.tensor(synth.extended_points(1, n)[..., 0], dtype=torch.float64, device="cuda")
        r2 = x * x
        for _ in range(d - 1):
            r2 = r2.unsqueeze(-1) + (x * x)
        G = torch.exp(-r2).contiguous()
        del x, r2
        b = torch.empty((n,) * d, dtype=torch.float64, device="cuda")
        op.boundary(G, out=b)
        barrier()
        t0 = time.perf_counter()
        for _ in range(3):
            op.boundary(G, out=b)
        barrier()
        ms = (time.perf_counter() - t0) / 3 * 1e3
        N = n + 1
        E = 3 * N - 1
        Mp = 1 << (E - 1).bit_length()
        if d == 1:
            flops = 2.0 * n * (2 * N + 1)
        else:
            Kp = Mp // 2 + 1
            lines = E + 2 * Kp + n if d == 2 else E * E + Kp * E + 2 * Kp * Mp + Kp * n + n * n
            flops = lines * 5.0 * Mp * math.log2(Mp)
        out[name] = {"ms": ms, "fft_side": Mp if d > 1 else None, "nominal_fp64_gflops": flops / (ms * 1e-3) / 1e9}
        op.close()
        del G, b
    return out


def build_measurement(fg, barrier) -> dict:
    """Operator build (frac_coeffs: weights, stencil, centre, symbol, tau symbol;
    synchronous) for the sizes of the served stream, alpha = 1.3, lambda in {0, 1}:
    ms of the second of two builds, host clock around the call."""
    out = {}
    for d, n, p in ((3, 63, 1), (3, 127, 1), (3, 255, 0), (3, 255, 1), (3, 255, 2), (2, 511, 2), (2, 1023, 2),
                    (1, 4095, 2)):
        for lam in (0.0, 1.0):
            ms = 0.0
            for _ in range(2):
                barrier()
                t0 = time.perf_counter()
                op = fg.FracOp(d, n, 1.3, degree=p, lam=lam)
                barrier()
                ms = 1e3 * (time.perf_counter() - t0)
                op.close()
            out[f"{d}d_n{n}_p{p}_lam{lam:g}"] = ms
    return out


def batch_measurement(fg, torch, barrier, fft: str = "pow2") -> dict:
    """256 mixed problems (d in {1, 2}, 1D n in [63, 4095], 2D side in [63, 511],
    alpha ~ U(0.1, 1.9), p in {0, 1, 2}, lambda ~ U(0, 2), smooth random right-hand
    sides) solved by one frac_solve_batch call, FP32 CG in FP64 refinement to 1e-10:
    1D problems one block each (one launch per FFT length), 2D problems of
    power-of-two lengths in one persistent cluster launch (mixed lengths, with fft
    "auto" or "smooth", through the solve engine).  The warm-up batch holds one
    problem of every FFT length, so the autotuner's one-time timings fall outside the
    timed call."""
    probs = synth.batch_problems(256)
    t0 = time.perf_counter()
    ops = [fg.FracOp(p.d, p.n, p.alpha, degree=p.degree, lam=p.lam, fft=fft) for p in probs]
    barrier()
    t_coeff = time.perf_counter() - t0
    fs = [torch.tensor(synth.smooth_field(p.d, p.n, p.seed) + 0.25, device="cuda") for p in probs]
    us = [torch.empty_like(f) for f in fs]
    classes = {}
    for i, p in enumerate(probs):
        classes.setdefault((p.d, ops[i].info()["fft_len"]), i)
    warm = sorted(classes.values())
    t0 = time.perf_counter()
    fg.solve_batch([ops[i] for i in warm], [fs[i] for i in warm], [us[i] for i in warm])
    barrier()
    t_warm = time.perf_counter() - t0
    t0 = time.perf_counter()
    infos = fg.solve_batch(ops, fs, us, rtol=1e-10, precision="mixed")
    barrier()
    dt = time.perf_counter() - t0
    plan = fg.batch_last_plan()
    dof = sum(p.n ** p.d for p in probs)
    ok = sum(1 for i in infos if i["status"] == 0 and i["rel_resid"] <= 1e-10)
    mixed = sum(1 for op in ops if any(m & (m - 1) for m in op.info()["fft_lens"]))
    for op in ops:
        op.close()
    return {"problems": len(probs), "fft_lengths": fft, "mixed_length_problems": mixed, "converged": ok,
            "solves_per_s": len(probs) / dt, "ms": 1e3 * dt,
            "dof_total": dof, "iters_total": int(sum(i["iters"] for i in infos)),
            "coefficient_build_ms_all_ops": 1e3 * t_coeff, "warmup_incl_autotune_ms": 1e3 * t_warm,
            "persistent_2d_plan": plan}


def _served_requests(fg, probs, arr):
    from paper_2103_03658_gb300 import serve
    pool = {}
    reqs = []
    for i, (pb, t) in enumerate(zip(probs, arr)):
        key = (pb.d, pb.n, i % 2)
        if key not in pool:
            pool[key] = synth.smooth_field(pb.d, pb.n, 7000 + len(pool)) + 0.25
        reqs.append(serve.Request(i, pb.d, pb.n, pb.alpha, pb.degree, pb.lam, pool[key], float(t)))
    return reqs


def _serve(fg, reqs, barrier, realtime=True, precision="mixed") -> tuple:
    from paper_2103_03658_gb300 import serve
    srv = serve.Server(hbm_budget=150e9, nstreams=16, precision=precision)
    barrier()
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=realtime)
    wall = time.perf_counter() - t0
    srv.close()
    return res, wall, srv


def _oracle_residual(args):
    """The oracle's relative residual ||f - A u|| / ||f|| of one served result, A built
    from the oracle's own generator: over every row in 1D, over 64 seeded rows otherwise."""
    from oracle import frac_oracle as O
    d, n, alpha, degree, lam, f, u = args
    N = n + 1
    a = O.stencil(d, N, 2.0 / N, alpha, degree, lam, q=20 if d < 3 else 12)
    c = O.c_dalpha(d, alpha)
    if d == 1:
        r = f - O.apply_dense(a, c, u)
        return float(np.linalg.norm(r) / np.linalg.norm(f))
    rows = np.random.default_rng(n).integers(0, n, size=(64, d))
    fr = f[tuple(rows.T)]
    return float(np.linalg.norm(fr - O.apply_rows(a, c, u, rows)) / np.linalg.norm(fr))


def oracle_sample(reqs, res, every: int = 50, max_nd: int = 63 ** 3) -> dict:
    """Every `every`-th served request (the next one whose oracle generator takes seconds,
    n^d <= 63^3, when the due one is larger) checked by the oracle on the host cores."""
    import multiprocessing as mp
    byid = {r.rid: r for r in res}
    picks, due = [], 0
    for q in reqs:
        if q.rid >= due and q.n ** q.d <= max_nd and q.rid in byid:
            picks.append(q)
            due = q.rid + every
    jobs = [(q.d, q.n, q.alpha, q.degree, q.lam, np.asarray(q.f, dtype=np.float64),
             np.asarray(byid[q.rid].u, dtype=np.float64)) for q in picks]
    if not jobs:
        return {"checked": 0}
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        errs = pool.map(_oracle_residual, jobs)
    by_d = {}
    for q, e in zip(picks, errs):
        by_d.setdefault(str(q.d), []).append(e)
    return {"checked": len(jobs), "every": every, "max_rel_resid": max(errs), "median_rel_resid": float(np.median(errs)),
            "max_rel_resid_by_d": {k: max(v) for k, v in sorted(by_d.items())},
            "rows": "all rows (1D), 64 seeded rows (2D, 3D)"}


def served_measurement(fg, torch, barrier, seconds: float = 2.0) -> dict:
    """Poisson arrivals at 200 req/s for `seconds`: d in {1, 2, 3} (0.4/0.4/0.2),
    1D/2D sizes as in the batch mix, 3D side in {63, 127, 255}, alpha ~ U(0.1, 1.9),
    lambda ~ U(0, 2), p in {0, 1, 2}; right-hand sides drawn from a seeded pool of
    two smooth fields per grid; 150 GB admission budget; latency from arrival to
    the solution on the host.  Reported for the fresh mix (every request a new
    operator) and the repeat mix (80 % of requests from 16 fixed problems), with
    the offered load rho = arrival rate / completed rate when the window ends
    with work still queued, and mixed vs plain FP64 solves/s on the first 48
    requests served back to back."""
    from paper_2103_03658_gb300 import serve
    arr = synth.arrival_times(rate=200.0, duration=seconds)
    out = {}
    for name, probs in (("fresh", synth.served_problems(len(arr))), ("repeat", synth.served_problems_repeat(len(arr)))):
        reqs = _served_requests(fg, probs, arr)
        res, wall, srv = _serve(fg, reqs, barrier)
        lat = [r.latency_s for r in res]
        ok = sum(1 for r in res if r.info["status"] == 0 and r.info["rel_resid"] <= 1e-10)
        by_d = {}
        for r, q in zip(res, reqs):
            by_d.setdefault(q.d, []).append(r.latency_s)
        rate_done = len(res) / wall
        check = oracle_sample(reqs, res)
        out[name] = {"requests": len(reqs), "window_s": seconds, "rate_per_s": 200.0, "converged": ok,
                     "oracle_check": check,
                     "solves_per_s": rate_done, "wall_s": wall,
                     "rho": (200.0 / rate_done) if wall > 1.2 * seconds else None,
                     "p50_ms": 1e3 * serve.percentile(lat, 50), "p99_ms": 1e3 * serve.percentile(lat, 99),
                     "p50_ms_by_d": {str(d): 1e3 * serve.percentile(v, 50) for d, v in sorted(by_d.items())},
                     "p99_ms_by_d": {str(d): 1e3 * serve.percentile(v, 99) for d, v in sorted(by_d.items())},
                     "op_cache_hits": srv.cache.hits, "op_cache_misses": srv.cache.misses}
    probs = synth.served_problems(48)
    reqs = _served_requests(fg, probs, np.zeros(len(probs)))
    cmp = {}
    for prec in ("mixed", "f64"):
        res, wall, _ = _serve(fg, reqs, barrier, realtime=False, precision=prec)
        ok = sum(1 for r in res if r.info["status"] == 0 and r.info["rel_resid"] <= 1e-10)
        cmp[prec] = {"solves_per_s": len(res) / wall, "wall_s": wall, "converged": ok}
    out["first48_back_to_back"] = cmp
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fields", type=int, default=65,
                    help="fields per apply (65 = the benchmark workload; fewer only for profiler captures)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 256-problem batch measurement and print its JSON (profiler captures)")
    ap.add_argument("--boundary-only", action="store_true",
                    help="run only the frac_boundary timings and print their JSON (profiler captures)")
    ap.add_argument("--served-only", action="store_true",
                    help="run only the served-stream measurement and print its JSON")
    ap.add_argument("--served-seconds", type=float, default=2.0,
                    help="arrival window of the served stream (the configured stream is 60 s)")
    ap.add_argument("--applies-only", action="store_true",
                    help="run only the 1D and 3D single-vector apply timings and print their JSON (profiler captures)")
    ap.add_argument("--precond-only", action="store_true",
                    help="run only the tau preconditioner timings and print their JSON (profiler captures)")
    ap.add_argument("--mixed-only", default=None, metavar="CASES",
                    help="run only the mixed-radix comparison for the listed cases (comma-separated, e.g. "
                         "2d_n600_b64; 'all' for every case) and print its JSON (profiler captures)")
    ap.add_argument("--batch-fft", default="pow2", choices=["pow2", "smooth", "auto"],
                    help="FFT-length policy of the operators of --batch-only")
    args = ap.parse_args()
    global NFIELDS
    NFIELDS = args.fields
    if args.applies_only:
        import torch
        import paper_2103_03658_gb300 as fg
        print(json.dumps(apply_measurement(fg, torch, torch.cuda.synchronize)), flush=True)
        return
    if args.precond_only:
        import torch
        import paper_2103_03658_gb300 as fg
        print(json.dumps(precond_measurement(fg, torch, torch.cuda.synchronize)), flush=True)
        return
    if args.boundary_only:
        import torch
        import paper_2103_03658_gb300 as fg
        print(json.dumps(boundary_measurement(fg, torch, torch.cuda.synchronize)), flush=True)
        return
    if args.served_only:
        import torch
        import paper_2103_03658_gb300 as fg
        print(json.dumps(served_measurement(fg, torch, torch.cuda.synchronize, args.served_seconds)), flush=True)
        return
    if args.batch_only:
        import torch
        import paper_2103_03658_gb300 as fg
        print(json.dumps(batch_measurement(fg, torch, torch.cuda.synchronize, fft=args.batch_fft)), flush=True)
        return
    if args.mixed_only:
        import torch
        import paper_2103_03658_gb300 as fg
        cases = None if args.mixed_only == "all" else set(args.mixed_only.split(","))
        print(json.dumps(mixed_radix_measurement(fg, torch, torch.cuda.synchronize, cases)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

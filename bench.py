"""FDiRW hot-path benchmark on GB300.

One benchmark step is one pass of the whole hot path over one synthetic workload:
  fdirw_create   -- face conductances and stability check
  fdirw_kernels  -- per-source windowed FD march + FP64 renormalisation (kernel cache)
  fdirw_step     -- `macro_steps` superposition steps and the FP64 mass budget
Metric: macro-steps/s of that job (the kernel build is amortised over the workload's macro steps),
timed with CUDA events on the stream the library launches on, inputs resident in HBM.  Extra keys give
source-kernels/s (march kernel alone) and the steady-state macro-steps/s (gather + scale per step).

  python bench.py [--steps K] [--warmup W] [--workload fdirw-192c-r8] [--prec bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores, bounded samples
  torchrun --nproc-per-node N bench.py --gpus N   # N independent replicas (one per GPU), weak scaling
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FDiRW macro-steps/sec at 192³ and source-kernels/sec vs plain FP64 GPU at ≤1e-5 rel L2"
UNIT = "macro-steps/s"
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (Blackwell)
FLOP_PER_CELL_SUBSTEP = 13       # coefficient form of the 7-point update: 1 MUL + 6 FMA
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The largest of every rank's time (all ranks get it); identity without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return world_size * units_per_rank * 1000.0 / max_ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- oracle (CPU) timing

def oracle_sample(w, D, n_sources: int, seed: int = 7, threads: int = 0):
    """Times the FP64 CPU oracle's kernel marches on a seeded sample of sources (all host threads unless
    `threads` is given).  The oracle recomputes every source's kernel for each superposition step, so one
    of its macro steps costs N kernel marches; the sample gives seconds per source."""
    import oracle
    shape = (w.n,) * 3
    lam = oracle.stable_dt_sub(shape, D)
    cond = oracle.Conductance(shape, D)
    rng = np.random.default_rng(seed)
    src = rng.integers(0, w.n ** 3, n_sources)
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.kernels(shape, D, lam, w.R, w.n_sub, src, cond)
    dt = time.perf_counter() - t0
    return dt / n_sources, threads, dt


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.strip().lower().startswith("model name"):
                return l.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith("model name"):
                return l.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_single_thread(w, D, n_sources: int, seed: int = 11):
    """Seconds per source of the FP64 oracle on ONE host thread (seeded sample), for the single-core figure."""
    import oracle
    t_src, _, dt = oracle_sample(w, D, n_sources, seed, threads=1)
    oracle.set_threads(os.cpu_count() or 1)
    return t_src, dt


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    _, D, _ = w.make()
    N = w.n ** 3
    per_step = []
    for i in range(args.warmup + args.steps):
        t_src, threads, _ = oracle_sample(w, D, args.ref_sample, seed=100 + i)
        if i >= args.warmup:
            per_step.append(t_src)
    t_src = statistics.mean(per_step)
    value = 1.0 / (N * t_src)
    t1, dt1 = oracle_single_thread(w, D, args.ref_sample_1t)
    sample = (f"{args.ref_sample} seeded random sources of {w.name} per step (FP64 windowed marches); "
              f"macro-steps/s = 1/(N * seconds per source), the oracle recomputing every kernel each step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * N * t_src, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": f"{w.n}^3", "R": w.R, "n_sub": w.n_sub,
                       "macro_steps": w.steps, "prec": "fp64", "accum": "fp64"},
            "timing": {"kind": "sample-extrapolated", "sources_per_step": args.ref_sample,
                       "timed_ms_per_step": 1000.0 * args.ref_sample * t_src,
                       "note": "each step times the sample; ms_per_step and value extrapolate it to all N sources"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(),
                             "single_thread": {"value": 1.0 / (N * t1), "cores": 1,
                                               "sample": f"{args.ref_sample_1t} seeded random sources ({dt1:.1f} s)"}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- CUDA path

def march_kernel_name(prec: str, parts: int) -> str:
    if prec == "fp64":
        return "march_f64_kernel<R>"
    return {4: "march_tm_kernel<R>", 5: "march_tmc_kernel<R>", 6: "march_tmp_kernel<R>", 7: "march_tmx_kernel<R>"}.get(
        parts, f"march_f32_kernel<R,{parts}>")


# DRAM bytes (read + write) per clipped window cell of march_tm_kernel<8> with BF16 storage, from one ncu
# capture of the 64^3 case with the same recipe (`--set full` on the first march launch of `bench.py
# --workload fdirw-64c-r8 --prec bf16 --march-parts 4 --no-surrogate --no-probe`: 0.641 GB read + 2.307 GB
# written over 1.0488e9 window cells); the traffic of a full launch scales with its window cells (the
# stored kernel values dominate it).  Valid for that kernel, radius and storage only.
TM_R8_BF16_DRAM_BYTES_PER_WINDOW_CELL = (0.641067008e9 + 2.306592e9) / 1048772096


def march_traffic(args, prec: str, parts: int, R: int, window_cells: float):
    if args.traffic is not None:
        return args.traffic
    if prec == "bf16" and parts == 4 and R == 8:
        return TM_R8_BF16_DRAM_BYTES_PER_WINDOW_CELL * window_cells
    return None


# DRAM bytes (read + write) per algorithmic byte of gather_fp32_kernel<bf16> from one ncu capture of the
# 96^3, R = 6 case (`bench.py --workload fdirw-96c-r6`: 3.8927e9 read + 3.33e6 written against
# 3.8971e9 algorithmic); the traffic of a launch grows with its cache bytes.  Valid for that kernel and
# storage only.
GATHER_FP32_BF16_DRAM_PER_ALGORITHMIC_BYTE = (3.892684288e9 + 3.326464e6) / (96 ** 3 * (13 ** 3 * 2 + 4 + 8))


def gather_roofline(prec: str, accum: str, N: int, R: int, gather_ms: float, probe=None):
    """HBM roofline of one superposition launch: algorithmic bytes = the kernel cache (N (2R+1)^3 stored
    values, each read once) + the scaled field it multiplies (FP32, or FP32 pairs) + the FP64 output."""
    peaks, peak_src = _peaks()
    qb = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[prec]
    chat_b = 8 if prec == "fp64" else (4 if accum == "fp32" else 8)
    nbytes = N * (2 * R + 1) ** 3 * qb + N * chat_b + N * 8
    achieved = nbytes / (gather_ms * 1e-3) / 1e9
    kname = ("gather_f64_kernel<R>" if prec == "fp64" else
             "gather_fp32_kernel<ST,R>" if accum == "fp32" else "gather_ff_kernel<ST,R>")
    traffic = GATHER_FP32_BF16_DRAM_PER_ALGORITHMIC_BYTE * nbytes if (prec == "bf16" and accum == "fp32") else None
    return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "traffic_source": "ncu capture of the 96^3 R=6 case of the same kernel and storage, DRAM bytes "
                              "scaled by algorithmic bytes to this launch" if traffic is not None else None,
            "peak_source": f"hbm_gbs ({peak_src}, a read + write copy)",
            "algorithmic": f"cache {N}x{(2 * R + 1) ** 3}x{qb} B + field {chat_b} B + output 8 B per cell "
                           f"= {nbytes / 1e9:.2f} GB per launch",
            **({"read_peak_measured": probe["read_bytes_per_s"] / 1e9,
                "frac_of_read_peak": achieved / (probe["read_bytes_per_s"] / 1e9),
                "read_peak_source": "measured in this run: streaming read of a 4 GiB buffer (fdirw_probe_peaks); the "
                                    "gather reads almost only, so this is its tighter ceiling"} if probe else {})}


def fp32_alu_roofline(torch, dev, n_sub: int, window_cells: float, march_ms: float, traffic, clocks, kname: str,
                      probe=None):
    """Achieved FP32 flop rate of the march (13 flop per cell-substep over the clipped windows) against the
    FP32 FMA rate measured on this GPU in this run (fdirw_probe_peaks), beside the FP32 pipe's unit-count
    peak at the measured maximum SM clock."""
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    derived = num_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = FLOP_PER_CELL_SUBSTEP * n_sub * window_cells / (march_ms * 1e-3) / 1e12
    measured = probe["fp32_flops"] / 1e12 if probe else None
    peak = measured if measured else derived
    out = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic,
           "peak_source": ("measured in this run: FP32 FMA loop of fdirw_probe_peaks (register-only, 4 x 512 "
                           "threads per SM)" if measured else
                           f"derived: FP32 pipe, {num_sms} SMs x {FP32_LANES_PER_SM} FMA/clk x 2 flop x {sm_max:.0f} MHz"),
           "peak_derived": derived, "frac_of_derived": achieved / derived,
           "peak_derived_source": f"FP32 pipe: {num_sms} SMs x {FP32_LANES_PER_SM} FMA/clk x 2 flop x {sm_max:.0f} MHz "
                                  f"(sm_max_mhz, {peak_src})",
           "algorithmic": f"{FLOP_PER_CELL_SUBSTEP} flop per cell-substep x n_sub x sum of clipped window cells "
                          f"({window_cells:.4g})"}
    if clocks.get("sm_mhz"):
        out["frac_of_derived_at_sampled_clock"] = achieved / (num_sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    return out


# Shared-memory wavefronts of march_tm_kernel<8> per COMPUTED thread-cell-substep (every CTA batch marches 256
# threads x 68 cells whatever the windows' clipping), from the same 64^3 capture: 3.298e10 wavefronts over
# 87,382 batches x 256 x 68 x 200.  A launch's wavefronts scale with its computed cells; the shared-memory
# peak is one 128-byte wavefront per SM-cycle (32 banks x 4 B).
TM_R8_SMEM_WAVEFRONTS_PER_COMPUTED_CELL = 3.2981171846e10 / (87382 * 256 * 68 * 200)


def march_smem(n_src: int, n_sub: int, R: int, parts: int, march_ms: float, sm_mhz: float, num_sms: int):
    """Shared-memory throughput of the march launch as a fraction of one wavefront per SM-cycle (mapping 4
    at R = 8 only, the kernel the capture covers)."""
    if parts != 4 or R != 8:
        return None
    spb = 256 // (R + 1) ** 2
    computed = -(-n_src // spb) * 256 * 4 * (2 * R + 1) * n_sub
    wavefronts = TM_R8_SMEM_WAVEFRONTS_PER_COMPUTED_CELL * computed
    per_cycle = wavefronts / (march_ms * 1e-3 * sm_mhz * 1e6 * num_sms)
    return {"wavefronts_per_launch": wavefronts, "achieved_per_sm_cycle": per_cycle, "peak_per_sm_cycle": 1.0,
            "frac": per_cycle, "clock_mhz": sm_mhz,
            "source": "64^3 ncu capture of the same kernel (wavefronts per computed cell-substep), scaled to this "
                      "launch's computed cells; divided by its CUDA-event time at the sampled SM clock"}


def run_batch(args, bw):
    """The batched workload: every structure's radius map, kernels (chunk by chunk when they do not all
    fit) and all macro steps through one fdirw_create_batch context; one step = create + step + destroy."""
    import torch
    from paper_2408_11376_gb300 import build as libbuild
    from paper_2408_11376_gb300 import fdirw

    ws, rank, local = _dist()
    libbuild.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    t0 = time.perf_counter()
    shapes, Ds_host, cs_host = bw.make()
    t_gen = time.perf_counter() - t0
    Ds = [torch.from_numpy(D).to(dev) for D in Ds_host]
    c_host = np.concatenate(cs_host)
    N = c_host.size
    c0 = torch.from_numpy(c_host).to(dev)
    c1 = torch.empty_like(c0)
    stream = torch.cuda.Stream(device=dev)
    dt_sub = min(fdirw.fdirw_stable_dt(s, D, device=local) for s, D in zip(shapes, Ds))
    dt_macro = bw.n_sub * dt_sub
    prec = args.prec if args.prec != "fp64" else "bf16"

    def one_pass(times=None, p=prec, out=c1, acc=args.accum):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            ctx = fdirw.fdirw_create_batch(shapes, Ds, dt_macro, bw.R_min, bw.R_max, bw.n_sub, p, device=local,
                                           stream=stream, march_parts=args.march_parts, accum=acc)
            ev[1].record(stream)
            mass = fdirw.fdirw_step(ctx, c0, out, bw.steps, want_mass=True)
            ev[2].record(stream)
            info = fdirw.fdirw_get_info(ctx)
            fdirw.fdirw_destroy(ctx)
        if times is not None:
            stream.synchronize()
            times.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), info["kernels_ms"],
                          info["last_gather_ms"], mass, info))
        return mass

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    times = []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            one_pass(times)
        end.record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    total_ms = max_over_ranks(start.elapsed_time(end), pg, dev)
    info = times[-1][5]
    march_ms = statistics.mean(t[2] for t in times)
    gather_ms = statistics.mean(t[3] for t in times)
    mass0 = float(c_host.sum())

    e2e = None
    if not args.no_e2e:
        Dp = [torch.from_numpy(D).pin_memory() for D in Ds_host]
        cp = torch.from_numpy(c_host).pin_memory()
        op = torch.empty_like(cp).pin_memory()

        def e2e_pass():
            with torch.cuda.stream(stream):
                ctx = fdirw.fdirw_create_batch(shapes, Dp, dt_macro, bw.R_min, bw.R_max, bw.n_sub, prec,
                                               device=local, stream=stream, march_parts=args.march_parts,
                                               accum=args.accum)
                fdirw.fdirw_step(ctx, cp, op, bw.steps, want_mass=True)
                fdirw.fdirw_destroy(ctx)

        torch.cuda.synchronize(dev)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for _ in range(args.e2e_steps):
            e2e_pass()
        ee.record(stream)
        torch.cuda.synchronize(dev)
        e_ms = max_over_ranks(es.elapsed_time(ee) / args.e2e_steps, pg, dev)
        e2e = {"value": job_rate(ws, bw.steps, e_ms), "unit": UNIT, "h2d_bytes_per_step": 16 * N,
               "d2h_bytes_per_step": 8 * N + 8}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    accuracy = None
    if not args.no_fp64 and ws == 1 and prec != "fp32":
        ref = torch.empty_like(c0)
        one_pass(p="fp32", out=ref, acc="ff")
        stream.synchronize()
        accuracy = {"vs": "fp32 storage, float-float sums, same batch", "rel_l2": float((torch.linalg.vector_norm(c1 - ref) /
                                                                       torch.linalg.vector_norm(ref)).item())}
        del ref

    clocks = clk.summary()
    roofline = fp32_alu_roofline(torch, dev, bw.n_sub, info["window_cells"], march_ms, args.traffic, clocks,
                                 march_kernel_name(prec, info["march_parts"]))
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        t_src, threads, dt, ns = oracle_batch_sample(bw, shapes, Ds_host, dt_macro, args.ref_sample * 4)
        cpu = {"value": 1.0 / (N * t_src), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{ns} seeded random sources of {bw.name}, each on its own radius ({dt:.1f} s of FP64 "
                         f"windowed marches on {threads} host threads); macro-steps/s = 1/(N * seconds per source)"}
    nch = info["n_chunks"]
    n_launch = 5 * len(shapes) + 1 + nch * (2 + 2 * bw.steps) + 4
    if args.accum == "fp32":
        n_launch += 2 + 3 * nch * bw.steps       # structure totals, then the restoration per chunk and step
    value = job_rate(ws, bw.steps * args.steps, total_ms)
    n_src_pass = N
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": bw.name, "structures": len(shapes), "cells": N,
                   "sides": sorted(set(s[0] for s in shapes)), "R": f"{bw.R_min}..{bw.R_max} by rule",
                   "n_sub": bw.n_sub, "macro_steps": bw.steps, "prec": prec, "accum": args.accum,
                   "parallelism": "replicas" if ws > 1 else "single GPU", "chunks": nch,
                   "l2": f"inputs larger than L2 (kernel cache {info['cache_bytes'] / 1e9:.1f} GB per chunk)"},
        "source_kernels_per_s": n_src_pass / (march_ms * 1e-3),
        "phase_ms": {"create": statistics.mean(t[0] for t in times), "step_call": statistics.mean(t[1] for t in times),
                     "march_kernels": march_ms, "last_gather_per_chunk_sum": gather_ms, "host_generation_s": t_gen},
        "graph_launches_per_pass": info["graph_launches"],
        "mass_rel_err": abs(times[-1][4] - mass0) / mass0, "accuracy": accuracy,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": n_launch * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def oracle_batch_sample(bw, shapes, Ds, dt_macro, n_sources: int, seed: int = 9):
    """Seconds per source of the FP64 oracle on a seeded sample of the batch's sources, each marched on
    its own radius (all host threads)."""
    import oracle
    sizes = np.array([int(np.prod(s)) for s in shapes])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.integers(0, offs[-1], n_sources))
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    dt = 0.0
    for i, shape in enumerate(shapes):
        loc = pick[(pick >= offs[i]) & (pick < offs[i + 1])] - offs[i]
        if loc.size == 0:
            continue
        R = oracle.radius_map(Ds[i], dt_macro, 1.0, bw.R_min, bw.R_max)
        lam = dt_macro / bw.n_sub
        cond = oracle.Conductance(shape, Ds[i])
        for r in np.unique(R[loc]):
            sel = loc[R[loc] == r]
            t0 = time.perf_counter()
            oracle.kernels(shape, Ds[i], lam, int(r), bw.n_sub, sel, cond)
            dt += time.perf_counter() - t0
    return dt / n_sources, threads, dt, n_sources


def run_reference_batch(args, bw):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    shapes, Ds, _ = bw.make()
    N = sum(int(np.prod(s)) for s in shapes)
    dt_macro = bw.n_sub * min(oracle.stable_dt_sub(s, D) for s, D in zip(shapes, Ds))
    per_step = []
    for i in range(args.warmup + args.steps):
        t_src, threads, _, ns = oracle_batch_sample(bw, shapes, Ds, dt_macro, args.ref_sample * 4, seed=100 + i)
        if i >= args.warmup:
            per_step.append(t_src)
    t_src = statistics.mean(per_step)
    value = 1.0 / (N * t_src)
    sample = (f"{args.ref_sample * 4} seeded random sources of {bw.name} per step, each on its own radius; "
              "macro-steps/s = 1/(N * seconds per source), the oracle recomputing every kernel each step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * N * t_src, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": bw.name, "structures": len(shapes), "cells": N, "n_sub": bw.n_sub,
                       "macro_steps": bw.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, w):
    import torch
    from paper_2408_11376_gb300 import build as libbuild
    from paper_2408_11376_gb300 import fdirw

    ws, rank, local = _dist()
    libbuild.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    packing, D_host, c_host = w.make()
    shape = (w.n,) * 3
    N = w.n ** 3
    D = torch.from_numpy(D_host).to(dev)
    c0 = torch.from_numpy(c_host).to(dev)
    c1 = torch.empty_like(c0)
    stream = torch.cuda.Stream(device=dev)
    dt_sub = fdirw.fdirw_stable_dt(shape, D, device=local)
    dt_macro = w.n_sub * dt_sub
    prec = args.prec

    probe = None if args.no_probe else fdirw.fdirw_probe_peaks(local)

    def one_pass(times=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            ctx = fdirw.fdirw_create(shape, D, dt_macro, w.R, w.n_sub, prec, device=local, stream=stream,
                                       march_parts=args.march_parts, accum=args.accum)
            ev[1].record(stream)
            fdirw.fdirw_kernels(ctx)
            ev[2].record(stream)
            mass = fdirw.fdirw_step(ctx, c0, c1, w.steps, want_mass=True)
            ev[3].record(stream)
            info = fdirw.fdirw_get_info(ctx)
            fdirw.fdirw_destroy(ctx)
        if times is not None:
            stream.synchronize()
            times.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                          ev[0].elapsed_time(ev[3]), info["kernels_ms"], info["last_gather_ms"], mass, info))
        return mass

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    times = []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            one_pass(times)
        end.record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    total_ms = max_over_ranks(start.elapsed_time(end), pg, dev)
    info = times[-1][7]
    mass0 = float(np.sum(c_host))
    march_ms = statistics.mean(t[4] for t in times)
    gather_ms = statistics.mean(t[5] for t in times)
    steps_ms = statistics.mean(t[2] for t in times)

    # e2e through the C ABI with pinned host buffers: H2D of D and c, D2H of c' inside the timed region.
    e2e = None
    if not args.no_e2e:
        Dp = torch.from_numpy(D_host).pin_memory()
        cp = torch.from_numpy(c_host).pin_memory()
        op = torch.empty_like(cp).pin_memory()

        def e2e_pass():
            with torch.cuda.stream(stream):
                ctx = fdirw.fdirw_create(shape, Dp, dt_macro, w.R, w.n_sub, prec, device=local, stream=stream,
                                       march_parts=args.march_parts, accum=args.accum)
                fdirw.fdirw_step(ctx, cp, op, w.steps, want_mass=True)
                fdirw.fdirw_destroy(ctx)

        e2e_pass()
        torch.cuda.synchronize(dev)
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for _ in range(args.e2e_steps):
            e2e_pass()
        ee.record(stream)
        torch.cuda.synchronize(dev)
        e_ms = max_over_ranks(es.elapsed_time(ee) / args.e2e_steps, pg, dev)
        e2e = {"value": job_rate(ws, w.steps, e_ms), "unit": UNIT, "h2d_bytes_per_step": 16 * N,
               "d2h_bytes_per_step": 8 * N + 8}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    fp64, ref64 = None, None
    if not args.no_fp64 and ws == 1:
        fp64, ref64 = fp64_leg(fdirw, torch, dev, stream, w, shape, D, c0, dt_macro, value_prec=prec)

    clocks = clk.summary()
    roofline = fp32_alu_roofline(torch, dev, w.n_sub, info["window_cells"], march_ms,
                                 march_traffic(args, prec, info["march_parts"], w.R, info["window_cells"]), clocks,
                                 march_kernel_name(prec, info["march_parts"]), probe)
    roofline["smem"] = march_smem(N, w.n_sub, w.R, info["march_parts"], march_ms,
                                  clocks.get("sm_mhz") or _peaks()[0].get("sm_max_mhz", 2070.0),
                                  torch.cuda.get_device_properties(dev).multi_processor_count)
    if roofline["traffic"] is not None and args.traffic is None:
        roofline["traffic_source"] = ("ncu capture of the 64^3 case of the same kernel, radius and storage, DRAM "
                                      "bytes scaled by window cells to this launch")

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        t_src, threads, dt = oracle_sample(w, D_host, args.ref_sample)
        t1, dt1 = oracle_single_thread(w, D_host, args.ref_sample_1t)
        cpu = {"value": 1.0 / (N * t_src), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.ref_sample} seeded random sources of {w.name} ({dt:.1f} s of FP64 windowed marches "
                         f"on {threads} host threads); macro-steps/s = 1/(N * seconds per source), the oracle "
                         "recomputing every kernel each step",
               "cpu_model": cpu_model(),
               "single_thread": {"value": 1.0 / (N * t1), "cores": 1,
                                 "sample": f"{args.ref_sample_1t} seeded random sources ({dt1:.1f} s)"}}

    n_launch = 4 + 1 + 2 + 2 * w.steps + 2      # conductance + 3 coef, march, mass(in), scale+gather per step, mass(out)
    if args.accum == "fp32":
        n_launch += 2 + 3 * w.steps             # the input's FP64 total, then the mass restoration per step
    value = job_rate(ws, w.steps * args.steps, total_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": w.name, "grid": f"{w.n}^3", "R": w.R, "n_sub": w.n_sub, "macro_steps": w.steps,
                   "prec": prec, "accum": args.accum, "porosity": w.porosity,
                   "mass": ("FP64 total restored to the input's after every macro step (FP32 row sums are not "
                            "mass-neutral)" if args.accum == "fp32" else "float-float row sums; no restoration"),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "march_threads_per_column": info["march_parts"],
                   "l2": f"inputs larger than L2 (kernel cache {info['cache_bytes'] / 1e9:.1f} GB, read every step)"},
        "source_kernels_per_s": N / (march_ms * 1e-3),
        "steady_macro_steps_per_s": 1000.0 * w.steps / steps_ms,
        "phase_ms": {"create": statistics.mean(t[0] for t in times), "kernels": statistics.mean(t[1] for t in times),
                     "march_kernel": march_ms, "steps": steps_ms, "gather_kernel": gather_ms},
        "mass_rel_err": abs(times[-1][6] - mass0) / mass0,
        "mass_restoration": ({"enforced_every_step": True, "pre_restoration_drift_max": info["last_restore_drift"],
                              "note": "mass_rel_err is 0 by construction here; the drift is |M_in - S| / M_in of "
                                      "the FP32-accumulated field before each step's restoration"}
                             if args.accum == "fp32" else None),
        "roofline": roofline, "gather_roofline": gather_roofline(prec, args.accum, N, w.R, gather_ms, probe),
        "measured_peaks": probe,
        "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu_baseline": fp64,
        "gpu_launches": n_launch * args.steps, "clocks": clocks,
    }
    if fp64:
        line["speedup_vs_fp64_gpu"] = value / fp64["macro_steps_per_s"]
    if args.oracle_full_step:
        line["oracle_full_step"] = oracle_full_step_leg(fdirw, torch, stream, w, shape, D, D_host, c0, c_host, dt_macro,
                                                        prec, args.accum)
    if args.surrogate:
        line["surrogate"] = surrogate_leg(args, fdirw, torch, dev, stream, w, shape, D, c0, dt_macro, prec, ref64)
    if args.coarse:
        line["coarse_mesh"] = coarse_leg(args, fdirw, torch, dev, stream, w, shape, D, ~packing.solid, dt_macro)
    if args.flow:
        line["convection"] = flow_leg(args, fdirw, torch, dev, stream, w, shape, D, packing.solid, dt_macro)
    if args.coupled:
        line["coupled"] = coupled_leg(args, fdirw, torch, dev, stream, w, shape, D, ~packing.solid, dt_macro)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def oracle_full_step_leg(fdirw, torch, stream, w, shape, D, D_host, c0, c_host, dt_macro, prec, accum):
    """One complete macro step of the workload by the FP64 oracle on all host cores (every source's kernel
    marched on the CPU; the per-source-radius superposition with every radius = R, which the oracle's pins
    tie to the uniform one bit for bit), against the plain FP64 GPU path and the bench's precision."""
    import oracle
    N = c0.numel()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    ref = oracle.superpose_rmap(shape, D_host, dt_macro / w.n_sub, np.full(N, w.R, dtype=np.int32), w.n_sub, c_host)
    t_oracle = time.perf_counter() - t0
    refd = torch.from_numpy(ref).to(c0.device)
    out = {"oracle_s": t_oracle, "cores": threads, "cpu_model": cpu_model()}
    for p, acc in (("fp64", "ff"), (prec, accum)):
        with torch.cuda.stream(stream):
            ctx = fdirw.fdirw_create(shape, D, dt_macro, w.R, w.n_sub, p, stream=stream, accum=acc)
            got = torch.empty_like(c0)
            fdirw.fdirw_step(ctx, c0, got, 1)
            fdirw.fdirw_destroy(ctx)
        stream.synchronize()
        out[f"rel_l2_{p}_{acc}_vs_oracle"] = float((torch.linalg.vector_norm(got - refd) /
                                                    torch.linalg.vector_norm(refd)).item())
        del got
        torch.cuda.empty_cache()
    return out


def surrogate_leg(args, fdirw, torch, dev, stream, w, shape, D, c0, dt_macro, prec, ref64=None):
    """Learned surrogate: trains on FD kernels of seeded packings (porosity U[0.3,0.5], per-sphere log10
    ratio U[3,8]; 200k kernels by default), then builds the workload's kernel cache with the gate and FD
    fallback and compares it with the FD-only build: build times, the network's convolution time and
    tensor-core rate, per-source costs and the acceptance that would make the gated build break even,
    acceptance of solid and pore sources, the error of accepted kernels against FD, and the field after
    the workload's macro steps against the FD-only field and the plain FP64 field."""
    from paper_2408_11376_gb300 import surrogate as sg
    t0 = time.perf_counter()
    data = sg.training_set(args.surrogate_structures, args.surrogate_per_structure, 20240825, n_sub=w.n_sub)
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    net = fdirw.Net(sg.init_params(20240826))
    t0 = time.perf_counter()
    hist = sg.train(net, data, args.surrogate_epochs, batch=256, lr=args.surrogate_lr)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    n_train = sum(len(d.sources) for d in data)
    for d in data:
        d.ctx.close()
    del data
    torch.cuda.empty_cache()
    N = c0.numel()
    solid = (D < 0.5).cpu().numpy()
    rng = np.random.default_rng(5)
    probe = np.sort(rng.integers(0, N, 4096))
    res = {}
    for mode in ("fd", "surrogate"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            f = fdirw.FDiRW(shape, D, dt_macro, w.R, w.n_sub, prec, stream=stream)
            if mode == "fd":
                f.kernels()                    # warm the autotuner outside the timed build
                stream.synchronize()
            e0.record(stream)
            acc = f.kernels() if mode == "fd" else net.build_kernels(f.ctx)
            e1.record(stream)
            stream.synchronize()
            info = fdirw.fdirw_get_info(f.ctx)
            out = torch.empty_like(c0)
            mass = f.step(c0, out, w.steps, want_mass=True)
            k = f.read_kernels(probe)
            if mode == "surrogate":
                # the network's own rate: forward passes of 1024 sources, convolutions timed on the device
                src = rng.integers(0, N, 1024)
                net.predict(f.ctx, src)
                net.predict(f.ctx, src)
                conv_ms = net.conv_ms()
                # acceptance by phase on 16 batches of random sources
                samp = rng.integers(0, N, 16 * 1024)
                accs = np.concatenate([net.predict(f.ctx, samp[i:i + 1024])[2] for i in range(0, samp.size, 1024)])
            f.close()
        res[mode] = {"build_ms": e0.elapsed_time(e1), "accepted": acc if mode == "surrogate" else None,
                     "field": out, "mass": mass, "kernels": k, "march_ms": info["kernels_ms"]}
    sgm, fd = res["surrogate"], res["fd"]
    kd = np.linalg.norm((sgm["kernels"] - fd["kernels"]).reshape(len(probe), -1), axis=1)
    kn = np.linalg.norm(fd["kernels"].reshape(len(probe), -1), axis=1)
    changed = kd > 0
    mass0 = float(c0.sum().item())
    peaks, peak_src = _peaks()
    mma_flops = 1024 * 4 * 17 * 81 * 2 * 128 * 16 * 16      # 4 layers x 17 planes x 81 MMAs of 128 x 16 x 16
    useful = 27 * 2 * (7 * 16 + 16 * 16 + 16 * 16 + 16 * 1) * 17 ** 3
    net_us = conv_ms * 1e3 / 1024
    fd_us = fd["march_ms"] * 1e3 / N
    sa = solid[samp]
    out = {"training_kernels": n_train, "epochs": args.surrogate_epochs, "loss_per_epoch": hist,
           "data_gen_s": t_data, "train_s": t_train, "train_samples_per_s": n_train * len(hist) / t_train,
           "fd_build_ms": fd["build_ms"], "surrogate_build_ms": sgm["build_ms"],
           "gain_build": fd["build_ms"] / sgm["build_ms"],
           "accepted_fraction": sgm["accepted"] / N,
           "accepted_fraction_sample": {"solid": float(accs[sa].mean()) if sa.any() else None,
                                        "pore": float(accs[~sa].mean()) if (~sa).any() else None,
                                        "sources": int(samp.size)},
           "tensor": {"conv_ms_per_1024_sources": conv_ms, "mma_flops": mma_flops,
                      "achieved_tflops": mma_flops / (conv_ms * 1e-3) / 1e12,
                      "peak": peaks["bf16_tflops"], "frac": mma_flops / (conv_ms * 1e-3) / 1e12 / peaks["bf16_tflops"],
                      "peak_source": f"bf16_tflops ({peak_src})",
                      "useful_flops_per_source": useful},
           "per_source_us": {"fd_march": fd_us, "net_convolutions": net_us},
           "break_even_acceptance": net_us / fd_us,
           "probe_accepted_kernel_rel_l2": ({"max": float((kd / kn)[changed].max()), "median": float(np.median((kd / kn)[changed])),
                                             "n": int(changed.sum())} if changed.any() else None),
           "field_rel_l2_vs_fd_after_steps": float((torch.linalg.vector_norm(sgm["field"] - fd["field"]) /
                                                     torch.linalg.vector_norm(fd["field"])).item()),
           "mass_rel_err": abs(sgm["mass"] - mass0) / mass0}
    # one training step (forward, loss, tensor-core input and weight gradients, Adam) of 256 sources
    out["train_step"] = sg.train_rate(20, device=dev.index if dev.index is not None else 0)
    if ref64 is not None:
        out["field_rel_l2_vs_fp64_after_steps"] = float((torch.linalg.vector_norm(sgm["field"] - ref64) /
                                                          torch.linalg.vector_norm(ref64)).item())
    net.close()
    return out


def coarse_leg(args, fdirw, torch, dev, stream, w, shape, D, liquid, dt_macro):
    """Coarse-mesh FDiRW (Eqs. 10-15) on the same geometry: the liquid (pore) cells of each B^3 block form
    one node, R and n_sub as the fine path.  Times create + coarse matrix + all macro steps.  Accuracy: a
    Gaussian blob (sigma = 10 cells) on the liquid cells, against the fine windowed FDiRW of the same
    liquid phase (D = 0 in the non-liquid cells, which gives those faces zero conductance)."""
    B = args.coarse
    n = shape[0]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r2 = ((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2).reshape(-1)
    c_liq = torch.from_numpy(np.where(liquid, np.exp(-r2 / (2 * 10.0 ** 2)), 0.0)).to(dev)
    lq = torch.from_numpy(liquid.astype(np.uint8)).to(dev)
    runs = []
    for _ in range(3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        out = torch.empty_like(c_liq)
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            ctx = fdirw.fdirw_create_coarse(shape, D, lq, B, dt_macro, w.R, w.n_sub, args.prec, device=dev.index,
                                            stream=stream)
            ev[1].record(stream)
            fdirw.fdirw_kernels(ctx)
            ev[2].record(stream)
            mass = fdirw.fdirw_step(ctx, c_liq, out, w.steps, want_mass=True)
            ev[3].record(stream)
            info = fdirw.fdirw_get_info(ctx)
            fdirw.fdirw_destroy(ctx)
        stream.synchronize()
        runs.append((ev[0].elapsed_time(ev[3]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]), info, mass, out))
    job_ms, build_ms, steps_ms, info, mass, out = runs[-1]
    fine = torch.empty_like(c_liq)
    with torch.cuda.stream(stream):
        ctx = fdirw.fdirw_create(shape, D * lq.to(D.dtype), dt_macro, w.R, w.n_sub, args.prec, device=dev.index,
                                 stream=stream)
        fdirw.fdirw_step(ctx, c_liq, fine, w.steps)
        fdirw.fdirw_destroy(ctx)
    stream.synchronize()
    mass0 = float(c_liq.sum().item())
    lqb = lq.bool()
    # Far-field boundary (Eqs. 7, 10, 14): outer surface open onto V_far = the liquid volume, c_far = 0.
    V_far = float(liquid.sum())
    far = torch.empty_like(c_liq)
    fe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        f = fdirw.FDiRWCoarse(shape, D, lq, B, dt_macro, w.R, w.n_sub, args.prec, device=dev.index, stream=stream)
        f.far_field(V_far, 0.0)
        fe[0].record(stream)
        f.kernels()
        f.step(c_liq, far, w.steps)
        fe[1].record(stream)
        c_far = f.c_far()
        f.close()
    stream.synchronize()
    far_total = float(far.sum().item()) + V_far * c_far
    far_leg = {"V_far_cells": V_far, "c_far0": 0.0, "c_far_after": c_far,
               "near_field_mass_after": float(far.sum().item()),
               "total_rel_err": abs(far_total - mass0) / mass0, "matrix_pbc_and_steps_ms": fe[0].elapsed_time(fe[1])}
    # Convection on the coarse path (Sec. 5): the far field above plus the --flow leg's face velocities
    # (mean 0.03 along +x, noise 0.03, zero on faces touching non-liquid cells) and, as there, n_sub raised
    # by a tenth so that the diffusive part leaves room for the advective outflow.
    from paper_2408_11376_gb300 import synth
    vel = torch.from_numpy(synth.face_velocity(shape, w.seed + 40, (0.03, 0.0, 0.0), 0.03, ~liquid).reshape(-1)).to(dev)
    flow_out = torch.empty_like(c_liq)
    ff = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    n_sub_flow = -(-11 * w.n_sub // 10)
    with torch.cuda.stream(stream):
        f = fdirw.FDiRWCoarse(shape, D, lq, B, dt_macro, w.R, n_sub_flow, args.prec, device=dev.index, stream=stream)
        f.far_field(V_far, 0.0)
        try:
            f.set_velocity(vel)
            ff[0].record(stream)
            f.kernels()
            ff[1].record(stream)
            f.step(c_liq, flow_out, w.steps)
            ff[2].record(stream)
            flow_cfar = f.c_far()
            stream.synchronize()
            flow_leg = {"velocity": "mean 0.03 along +x, noise 0.03, 0 on non-liquid faces", "n_sub": n_sub_flow,
                        "matrix_and_pbc_ms": ff[0].elapsed_time(ff[1]), "steps_ms": ff[1].elapsed_time(ff[2]),
                        "total_rel_err": abs(float(flow_out.sum().item()) + V_far * flow_cfar - mass0) / mass0}
        except fdirw.FdirwError as e:       # reported, not fatal: the other legs stand
            flow_leg = {"error": str(e)}
        f.close()
    return {"block": B, "nodes": info["coarse_nodes"], "liquid_cells": int(liquid.sum()), "far_field": far_leg,
            "convection": flow_leg,
            "macro_steps_per_s": 1000.0 * w.steps / job_ms, "job_ms": job_ms, "matrix_build_ms": build_ms,
            "march_kernel_ms": info["kernels_ms"], "steps_ms": steps_ms,
            "march_cell_substeps_per_s": w.n_sub * info["window_cells"] / (info["kernels_ms"] * 1e-3),
            "matrix_bytes": info["cache_bytes"],
            "field": "Gaussian blob sigma 10 on the liquid cells",
            "rel_l2_vs_fine_liquid_phase": float((torch.linalg.vector_norm((out - fine)[lqb]) /
                                                  torch.linalg.vector_norm(fine[lqb])).item()),
            "mass_rel_err": abs(mass - mass0) / mass0}


def coupled_leg(args, fdirw, torch, dev, stream, w, shape, D, liquid, dt_macro):
    """Coupled macro step (Sec. 2): interface exchange, slow solid march and the coarse liquid FDiRW with
    the far field, on the workload's geometry (liquid = pore; the D map read as the effective D_m A_m/RT).
    Kinetics in lattice units chosen so that no face moves more than a percent of its liquid cell per step:
    k = 1e-7, cS_eq = 1, cL_eq = 1e-5; initial liquid 2.12e-3, solid 1e-6, far field 2.12e-3 over the
    liquid's volume (the proportions of the paper's Table 1)."""
    B = args.coarse or 5
    lq = torch.from_numpy(liquid.astype(np.uint8)).to(dev)
    c_init = torch.from_numpy(np.where(liquid, 2.12e-3, 1e-6)).to(dev)
    V_far = float(liquid.sum())
    cf0 = 2.12e-3
    field = c_init.clone()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(stream):
        f = fdirw.FDiRWCoarse(shape, D, lq, B, dt_macro, w.R, w.n_sub, args.prec, device=dev.index, stream=stream)
        f.far_field(V_far, cf0)
        ev[0].record(stream)
        f.kernels()
        ev[1].record(stream)
        QL, QS, c_far = f.coupled_step(field, w.steps, 1e-7, 1.0, 1e-5, dt_macro, 1)
        ev[2].record(stream)
        f.close()
    stream.synchronize()
    total0 = float(c_init.sum().item()) + V_far * cf0
    total = float(field.sum().item()) + V_far * c_far
    steps_ms = ev[1].elapsed_time(ev[2])
    return {"block": B, "macro_steps": w.steps, "matrix_and_pbc_ms": ev[0].elapsed_time(ev[1]),
            "steps_ms": steps_ms, "coupled_macro_steps_per_s": 1000.0 * w.steps / steps_ms,
            "Q_L": [QL[0], QL[-1]], "Q_S": [QS[0], QS[-1]], "c_far_after": c_far, "total_rel_err": abs(total - total0) / total0}


def flow_leg(args, fdirw, torch, dev, stream, w, shape, D, solid, dt_macro):
    """Convection (Sec. 5): a steady face-velocity field folded into every source's march (upwind faces,
    mapping 5), the superposition unchanged.  Flow: a mean of 0.03 cells per unit time along +x plus
    uniform noise of 0.03 on every face, zero on faces touching a solid cell; n_sub raised by a tenth so
    that the diffusive part leaves room for the advective outflow within the same macro step.  Field: a
    Gaussian blob (sigma 10 cells) on the pore cells.  Times create + velocity + kernels + macro steps
    with the flow, and the same n_sub on mapping 5 without it (the march's cost of the upwind faces)."""
    from paper_2408_11376_gb300 import synth
    n_sub = -(-11 * w.n_sub // 10)
    N = shape[0] * shape[1] * shape[2]
    vel = torch.from_numpy(synth.face_velocity(shape, w.seed + 40, (0.03, 0.0, 0.0), 0.03, solid).reshape(-1)).to(dev)
    n = shape[0]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r2 = ((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2).reshape(-1)
    c_in = torch.from_numpy(np.where(solid, 0.0, np.exp(-r2 / (2 * 10.0 ** 2)))).to(dev)
    xs = torch.from_numpy(x.reshape(-1).astype(np.float64)).to(dev)
    res = {}
    for flow in (True, False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        out = torch.empty_like(c_in)
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            ctx = fdirw.fdirw_create(shape, D, dt_macro, w.R, n_sub, args.prec, device=dev.index, stream=stream,
                                     march_parts=5)
            if flow:
                fdirw.fdirw_set_velocity(ctx, vel, N)
            ev[1].record(stream)
            fdirw.fdirw_kernels(ctx)
            ev[2].record(stream)
            mass = fdirw.fdirw_step(ctx, c_in, out, w.steps, want_mass=True)
            ev[3].record(stream)
            info = fdirw.fdirw_get_info(ctx)
            fdirw.fdirw_destroy(ctx)
        stream.synchronize()
        res[flow] = (ev[0].elapsed_time(ev[3]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]), info, mass,
                     float((out * xs).sum().item() / out.sum().item()))
    job_ms, build_ms, steps_ms, info, mass, xc = res[True]
    mass0 = float(c_in.sum().item())
    roof = fp32_alu_roofline(torch, dev, n_sub, info["window_cells"], info["kernels_ms"], None, {},
                             "march_tmc_kernel<R, ADV>")
    return {"n_sub": n_sub, "velocity": "mean 0.03 along +x, noise 0.03, 0 on solid faces",
            "macro_steps_per_s": 1000.0 * w.steps / job_ms, "job_ms": job_ms, "kernels_ms": build_ms,
            "steps_ms": steps_ms, "march_kernel_ms": info["kernels_ms"],
            "march_kernel_ms_no_flow_same_mapping": res[False][3]["kernels_ms"],
            "march_tflops": roof["achieved"], "march_frac_fp32": roof["frac"],
            "mass_rel_err": abs(mass - mass0) / mass0,
            "x_centroid_shift_vs_no_flow_cells": xc - res[False][5]}


def fp64_leg(fdirw, torch, dev, stream, w, shape, D, c0, dt_macro, value_prec):
    """The plain FP64 GPU FDiRW (FP64 march, FP64 cache, FP64 gather) run once over the workload, timed
    with CUDA events, keeping its field after every macro step; then every reduced-precision mode is run
    step by step and compared with it (relative L2 per step, and the mass budget)."""
    N = c0.numel()
    ref = torch.empty((w.steps, N), dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        ctx = fdirw.fdirw_create(shape, D, dt_macro, w.R, w.n_sub, "fp64", stream=stream)
        ev[1].record(stream)
        fdirw.fdirw_kernels(ctx)
        ev[2].record(stream)
        cur = c0
        for t in range(w.steps):
            fdirw.fdirw_step(ctx, cur, ref[t], 1)
            cur = ref[t]
        ev[3].record(stream)
        info = fdirw.fdirw_get_info(ctx)
        fdirw.fdirw_destroy(ctx)
    stream.synchronize()
    job_ms = ev[0].elapsed_time(ev[3])
    out = {"macro_steps_per_s": 1000.0 * w.steps / job_ms, "job_ms": job_ms,
           "source_kernels_per_s": N / (info["kernels_ms"] * 1e-3), "march_kernel_ms": info["kernels_ms"],
           "steps_ms": ev[2].elapsed_time(ev[3]), "cache_gb": info["cache_bytes"] / 1e9, "rel_l2_vs_fp64": {}}
    mass0 = float(c0.sum().item())
    out["mass_rel_err"] = abs(float(ref[-1].sum().item()) - mass0) / mass0
    for p, acc in (("fp32", "ff"), ("fp16", "ff"), ("bf16", "ff"), ("fp32", "fp32"), ("bf16", "fp32")):
        with torch.cuda.stream(stream):
            ctx = fdirw.fdirw_create(shape, D, dt_macro, w.R, w.n_sub, p, stream=stream, accum=acc)
            a = torch.empty_like(c0)
            errs = []
            cur = c0
            for t in range(w.steps):
                fdirw.fdirw_step(ctx, cur, a, 1)
                errs.append(float((torch.linalg.vector_norm(a - ref[t]) / torch.linalg.vector_norm(ref[t])).item()))
                cur = a.clone()
            m = fdirw.fdirw_mass(ctx, a)
            fdirw.fdirw_destroy(ctx)
        out["rel_l2_vs_fp64"][p if acc == "ff" else p + "_fp32acc"] = {
            "max_over_steps": max(errs), "last": errs[-1], "mass_rel_err": abs(m - mass0) / mass0}
    last = ref[-1].clone()
    del ref
    torch.cuda.empty_cache()
    return out, last


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="fdirw-192c-r8")
    ap.add_argument("--prec", choices=["fp64", "fp32", "fp16", "bf16"], default="bf16",
                    help="kernel-cache storage (BF16 meets 1e-5 rel L2 vs FP64 on fdirw-192c-r8, see the fp64 leg)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU baseline and accuracy leg")
    ap.add_argument("--surrogate", action="store_true",
                    help="train the learned surrogate and compare its gated build (on by default for R = 8 single grids)")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--oracle-full-step", action="store_true",
                    help="also run one complete macro step with the FP64 oracle on all host cores (about 15 min at "
                         "192^3) and compare the GPU's FP64 and default-precision steps with it")
    ap.add_argument("--surrogate-structures", type=int, default=20)
    ap.add_argument("--surrogate-per-structure", type=int, default=10000)
    ap.add_argument("--surrogate-epochs", type=int, default=4)
    ap.add_argument("--surrogate-lr", type=float, default=2e-3)
    ap.add_argument("--coarse", type=int, default=0,
                    help="also run the coarse-mesh FDiRW with this odd block side (e.g. 5) and compare it with the fine path")
    ap.add_argument("--coupled", action="store_true",
                    help="also run the coupled macro step (exchange, solid march, coarse FDiRW with far field)")
    ap.add_argument("--accum", choices=["ff", "fp32"], default="fp32",
                    help="superposition accumulation: float-float rows, or FP32 rows with the mass restored")
    ap.add_argument("--flow", action="store_true",
                    help="also time the convection path (steady face velocities folded into the march)")
    ap.add_argument("--ref-sample", type=int, default=32768, help="sources per oracle timing sample")
    ap.add_argument("--ref-sample-1t", type=int, default=2048, help="sources of the single-thread oracle sample")
    ap.add_argument("--march-parts", type=int, default=0,
                    help="force a march thread mapping (1-3 threads per column, 4 = 2x2 TMEM blocks, 5 = TMEM "
                         "lateral faces, 6 = source pairs in f32x2, 7 = column pairs with TMEM faces); 0 = autotune")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP32 FMA and HBM read peak probes")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per march launch from an ncu capture of the current kernel")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    from paper_2408_11376_gb300 import synth
    if args.prec == "fp64":
        args.accum = "ff"            # the FP64 path sums in FP64
    if args.workload in synth.BATCH_WORKLOADS:
        bw = synth.BATCH_WORKLOADS[args.workload]
        return run_reference_batch(args, bw) if args.impl == "reference" else run_batch(args, bw)
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if w.R == 8 and args.prec != "fp64" and not args.no_surrogate and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        args.surrogate = True
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())

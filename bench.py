"""Benchmark: r-RESPA with cutoff ATM three-body forces on one GB300 (arXiv 2507.11172).

Workload (default): 100,000 particles, FCC at density 0.8 with 0.05 sigma Gaussian jitter and
Maxwell velocities at T* = 1.0; LJ eps = sigma = 1, r_c = 2.5; ATM nu = 0.073, r_c = 2.5;
r-RESPA dt_outer = 0.02 with k = 10 inner steps.  One benchmark step = one outer r-RESPA step
(10 LJ evaluations with their velocity-Verlet updates, one binning sort + pair-list build, one
ATM evaluation, the outer kicks) through md_respa_step.

value = interacting triplets evaluated per second of whole-step time (FP32 forces with
compensated accumulation, FP64 integrator and energies).  Also reported: r-RESPA outer steps/s,
the same numbers for the all-FP64 path, the ATM kernel's roofline position, an end-to-end figure
through the C ABI with host buffers, and the CPU oracle on a bounded sample.

Multi-GPU (--gpus N under torchrun): independent replicas, one per rank (the method shards into
independent systems; there is no data-path collective), weak scaling; max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triplets/s and r-RESPA steps/s, FP32 vs FP64 plain; p50/p99 replica latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz maximum SM clock.  The
# roofline divides by the FMA throughput measured in the same run (md_measure_fma_peak); this figure
# is reported beside it.
FP32_PEAK_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic FP32 flops of one interacting triplet in the ATM kernel's formula (FMA = 2 flops),
# counted from atm_triplet: d_jk 3, c 5, ab/q 2, rsqrt 1 + Newton 4, w/t3/t5 3, s/A/B/C 8,
# AB/AC/BC/P 4, Pa/Pb/Pc 9, G 3, ia/ib/ic 5, nu*t5 1, pa2/pb2/pc2 12, F_i 9, F_j 9, F_k 3,
# accumulation of F_i (3) and scatter of F_j, F_k (6)
PROFILES = os.path.join(ROOT, "profiles")
# source files whose content decides each kernel's code: a profile's DRAM traffic counts only while
# their hash is the one recorded beside it
KERNEL_SOURCES = {
    "k_atm_rot<float>": ["paper_2507_11172_gb300/csrc/atm_rot.cu", "paper_2507_11172_gb300/csrc/md_internal.cuh"],
    "k_lj<float, 1>": ["paper_2507_11172_gb300/csrc/forces.cu", "paper_2507_11172_gb300/csrc/md_internal.cuh"],
}
ATM_FLOPS_PER_TRIPLET = 3 + 5 + 2 + 5 + 3 + 8 + 4 + 9 + 3 + 5 + 1 + 12 + 9 + 9 + 3 + 3 + 6


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` on the 100k workload from the ncu summary in
    profiles/ (a line `traffic: {json}` with the kernel, the bytes and the source hash at capture), or
    (None, reason) when there is none or the kernel's source has changed since."""
    import glob
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(path):
            line = line.strip()
            if not line.startswith("traffic: {"):
                continue
            rec = json.loads(line[len("traffic: "):])
            if rec.get("kernel") != kernel:
                continue
            if rec.get("source_sha256") != source_hash(kernel):
                return None, f"stale: {os.path.basename(path)} was captured from other source"
            return float(rec["dram_bytes_per_launch"]), os.path.basename(path)
    return None, "no capture in profiles/"


def measure_peaks(r3):
    """FP32 (plain and packed FMA) and FP64 FMA throughput of this GPU, with clock samples taken
    during the measurement (md_measure_fma_peak; each kind >= 60 ms per launch)."""
    stop, samples = threading.Event(), []
    th = threading.Thread(target=sample_clocks, args=(stop, samples), daemon=True)
    th.start()
    try:
        f32, _ = r3.md_measure_fma_peak(0, 60.0)
        f32x2, _ = r3.md_measure_fma_peak(1, 60.0)
        f64, _ = r3.md_measure_fma_peak(2, 60.0)
    finally:
        stop.set()
        th.join()
    return {"fp32_tflops": max(f32, f32x2) / 1e12, "fp32_ffma_tflops": f32 / 1e12, "fp32_ffma2_tflops": f32x2 / 1e12,
            "fp64_tflops": f64 / 1e12, "clocks": clock_summary(samples),
            "how": "md_measure_fma_peak: one full wave of resident CTAs, 8 independent FMA chains per thread, "
                   "best of 3 launches >= 60 ms (CUDA events)"}


def _nvml_sampler():
    """Read-only NVML queries through ctypes (SM clock, its maximum, clock-event reasons) for the GPU
    of this rank; None where the library is unavailable."""
    import ctypes
    try:
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(int(os.environ.get("LOCAL_RANK", "0")), ctypes.byref(h)) != 0:
            return None
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
    except (OSError, AttributeError):
        return None
    mx = ctypes.c_uint(0)
    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM

    def sample():
        c, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) != 0 or reasons_fn(h, ctypes.byref(r)) != 0:
            return None
        bits = (0x8, 0x40, 0x20, 0x4)  # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
        flags = ["Active" if r.value & b else "Not Active" for b in bits]
        return ", ".join([str(c.value), str(mx.value), "", hex(r.value)] + flags)
    return sample


def sample_clocks(stop, out):
    """Clock samples while the timed region runs: NVML every 10 ms, else nvidia-smi in a loop."""
    nv = _nvml_sampler()
    if nv is not None:
        while not stop.is_set():
            line = nv()
            if line:
                out.append(line)
            stop.wait(0.01)
        return
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", os.environ.get("LOCAL_RANK", "0")]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0:
                out.append(r.stdout.strip())
        except Exception:
            pass
        stop.wait(0.2)


def clock_summary(samples):
    sm, mx, reasons = [], None, set()
    for line in samples:
        f = [t.strip() for t in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            mx = float(f[1])
        except ValueError:
            continue
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for name, val in zip(names, f[4:8]):
            if val.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def workload(replica=0):
    import md_inputs
    return md_inputs.fcc_100k(replica)


def reduce_over_ranks(ms, units, device="cpu"):
    """(max over ranks of the timed region in ms, sum over ranks of the units processed); the
    identity without an initialised process group.  Works with any backend: pass the device the
    backend communicates on ("cuda" for NCCL, "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args):
    import torch
    import paper_2507_11172_gb300 as r3

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r3.load()
    peaks_run = measure_peaks(r3)
    fp32_peak = peaks_run["fp32_tflops"]
    w = workload(rank)  # weak scaling: every rank advances its own independent replica
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream()
    flush = torch.empty(int(256 * 2 ** 20) // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_passes(precision, steps, warmup):
        """Graph-replayed pass (the production path) for the step rate, then a profiled pass of
        the same number of steps (direct launches, CUDA events around each ATM launch on the
        library's stream) for the ATM kernel time."""
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, precision, stream.cuda_stream)
        try:
            r3.md_set_potentials(h, 1.0, 1.0, w.rc2, w.nu, w.rc3)
            if args.lj_kernel >= 0:  # pinned LJ kernel (row / cell-tile / team) instead of the autotuner's
                r3.md_set_lj_kernel(h, args.lj_kernel)
            with torch.cuda.stream(stream):
                r3.md_respa_step(h, 0, w.k_inner, w.dt_outer)  # initial forces F2b(x0), F3b(x0)
                for _ in range(warmup):
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                out = {}
                for profile in (False, True):
                    r3.md_set_profiling(h, profile)
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)  # build this mode's plan untimed
                    s0 = r3.md_get_stats(h)
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(steps)]
                    torch.cuda.synchronize()
                    barrier()
                    stop, samples = threading.Event(), []
                    th = threading.Thread(target=sample_clocks, args=(stop, samples), daemon=True)
                    th.start()
                    for e0, e1 in ev:
                        flush.fill_(1.0)  # L2 flush between steps (buffer larger than the 129 MB L2)
                        e0.record(stream)
                        r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                        e1.record(stream)
                    torch.cuda.synchronize()
                    stop.set()
                    th.join()
                    barrier()
                    s1 = r3.md_get_stats(h)
                    out[profile] = dict(ms=sum(e0.elapsed_time(e1) for e0, e1 in ev),
                                        trip=s1["triplets_total"] - s0["triplets_total"],
                                        atm_ms=(s1["atm_ms_total"] - s0["atm_ms_total"]),
                                        atm_n=s1["atm_timed"] - s0["atm_timed"], clocks=clock_summary(samples),
                                        kernel=s1["atm_kernel"], per=s1["atm_bases_per_warp"],
                                        tuned={k: s1[k] for k in ("atm_kernel", "atm_bases_per_warp", "lj_kernel",
                                                                   "lj_team", "lj_block", "list_warps")})
            return out
        finally:
            r3.md_destroy_system(h)

    p32 = timed_passes(r3.MD_FP32, K, W)
    g32, q32 = p32[False], p32[True]
    if q32["atm_n"] <= 0:
        raise RuntimeError("ATM kernel timing events were not recorded")
    ms32, trip32, clk = g32["ms"], g32["trip"], g32["clocks"]
    atm_ms = q32["atm_ms"] / q32["atm_n"]
    trip_per_eval = trip32 / K
    k64 = max(3, K // 4)
    p64 = timed_passes(r3.MD_FP64, k64, 3)
    ms64, trip64 = p64[False]["ms"], p64[False]["trip"]
    atm64_ms = p64[True]["atm_ms"] / max(1, p64[True]["atm_n"])

    # whole job: units of all ranks over the slowest rank's timed region
    t_local, trip_all = reduce_over_ranks(ms32, trip32, "cuda")
    value = trip_all / (t_local / 1e3)
    steps_per_s = K * world / (t_local / 1e3)

    # end to end through the C ABI with host buffers: per step the caller's state goes host->device,
    # one outer step runs, and the new state comes back device->host
    e2e = None
    if rank == 0:
        import ctypes
        n = w.n
        hx = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        hv = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        hx[:] = w.x
        hv[:] = w.v
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32, stream.cuda_stream)
        try:
            r3.md_set_potentials(h, 1.0, 1.0, w.rc2, w.nu, w.rc3)
            with torch.cuda.stream(stream):
                for _ in range(2):
                    r3.md_set_state(h, hx, hv)
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                    r3.md_get_state(h, hx, hv)
                ke = max(3, K // 4)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(ke):
                    r3.md_set_state(h, hx, hv)
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                    r3.md_get_state(h, hx, hv)
                torch.cuda.synchronize()
                te = time.perf_counter() - t0
            e2e = {"value": trip_per_eval * ke / te, "unit": "triplets/s", "h2d_bytes_per_step": 48 * n,
                   "d2h_bytes_per_step": 48 * n,
                   "note": "per step: md_set_state (host x, v) + md_respa_step(1 outer) + md_get_state; "
                           "set_state invalidates cached forces, so each step also re-evaluates F2b, F3b"}
        finally:
            r3.md_destroy_system(h)
        del ctypes

    # observables (Sec. 4.2.2): RDF pair counts over the pair list of the final positions (100 bins
    # up to r_c2), timed through the C ABI call (synchronous)
    obs_line = None
    if rank == 0:
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32, stream.cuda_stream)
        try:
            r3.md_set_potentials(h, 1.0, 1.0, w.rc2, w.nu, w.rc3)
            r3.md_get_rdf(h, 100, w.rc2)
            t0 = time.perf_counter()
            for _ in range(5):
                cnt = r3.md_get_rdf(h, 100, w.rc2)
            rdf_ms = (time.perf_counter() - t0) / 5 * 1e3
            obs_line = {"rdf_call_ms": rdf_ms, "rdf_pairs_below_rc": int(cnt.sum()), "rdf_bins": 100}
        finally:
            r3.md_destroy_system(h)

    classes_line = run_classes(r3, w, stream, flush, K) if rank == 0 else None
    w2m = large_workload() if (rank == 0 and not args.no_large) else None
    large_line = run_large(r3, stream, flush, *w2m) if w2m else None
    direct_line = run_direct(r3, stream, fp32_peak) if rank == 0 else None

    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    achieved_tflops = trip_per_eval * ATM_FLOPS_PER_TRIPLET / (atm_ms / 1e3) / 1e12
    kname = {0: "k_atm<float>", 1: "k_atm_pa<float>", 2: "k_atm_rot<float>"}.get(q32["kernel"])
    traffic, traffic_src = profiled_traffic(kname) if kname in KERNEL_SOURCES else (None, "no capture")
    fp64_tflops = trip64 / k64 * ATM_FLOPS_PER_TRIPLET / (atm64_ms / 1e3) / 1e12 if atm64_ms > 0 else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "triplets/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": t_local / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 forces (LJ sums compensated by TwoSum, ATM sums in exact 64-bit fixed point), "
                 "f64 integrator and energies",
        "data": "synthetic",
        "config": {"workload": "fcc100k_rho0.8: N=100000 FCC+jitter 0.05, LJ rc 2.5, ATM nu 0.073 rc 2.5, "
                               "r-RESPA k=10 dt_outer=0.02, one step = one outer step",
                   "n_particles": w.n, "box_L": w.L, "k_inner": w.k_inner, "dt_outer": w.dt_outer,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "rrespa_steps_per_s": steps_per_s,
        "triplets_per_atm_eval": trip_per_eval,
        "fp64_plain": {"triplets_per_s": trip64 / (ms64 / 1e3), "rrespa_steps_per_s": k64 / (ms64 / 1e3),
                       "atm_kernel_ms": atm64_ms, "atm_achieved_tflops": fp64_tflops,
                       "atm_frac_of_measured_fp64_peak": (fp64_tflops / peaks_run["fp64_tflops"]
                                                          if fp64_tflops and peaks_run["fp64_tflops"] > 0 else None)},
        "atm_kernel_ms": atm_ms,
        "profiled_pass_ms_per_step": q32["ms"] / K,
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp32_peak,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "kernel": kname,
                     "bases_per_warp": q32["per"] if q32["kernel"] == 2 else None,
                     "peak_source": "measured in this run (md_measure_fma_peak, FP32 FMA)",
                     "peak_nominal": FP32_PEAK_NOMINAL_TFLOPS,
                     "frac_of_nominal": achieved_tflops / FP32_PEAK_NOMINAL_TFLOPS,
                     "note": f"{ATM_FLOPS_PER_TRIPLET} flop per interacting triplet (FMA = 2) x interacting "
                             "triplets per launch / CUDA-event launch time; nominal peak = 152 SM x 128 FP32 "
                             "lanes x 2 x 2.07 GHz"},
        # the autotuner's choices for the timed system (LJ kernel 0 row, 1 cell tile, 2 team of lj_team
        # lanes per particle; triplet kernel 2 rotation with atm_bases_per_warp bases per warp)
        "autotuned": q32["tuned"],
        "fma_peaks": peaks_run,
        "clocks": clk,
        # per outer step: 2 LJ-phase launches (forces, kick/drift) per inner step, the sort (bin, scan,
        # cell order (2), scatter, listbuild), the triplet kernel and the combine; plus the opening
        # kick of each call
        "gpu_launches": K * (2 * w.k_inner + 8 + 1),
        "e2e": e2e,
        "observables": obs_line,
        "distance_classes": classes_line,
        "direct_sum": direct_line,
        "large_2m": large_line,
    }
    if peaks:
        line["measured_peaks"] = {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops")}
    if rank == 0 and not args.no_batch:
        line["ensemble"] = run_ensemble(r3)
        line["serving"] = run_serving(r3, seconds=args.serve_seconds, max_particles=args.serve_max_particles)
        # below capacity (about 25 requests/s of this mix on one GB300): latencies without queueing
        line["serving_subcapacity"] = run_serving(r3, seconds=5.0, rate=12.0, max_particles=args.serve_max_particles)
    if not args.no_cpu and rank == 0:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_sample)
        line["cpu_linked_cell"] = cpu_linked_cell(w, w2m[0] if w2m else None)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def large_workload():
    """The 2,000,000-particle random-sequential-addition start and the seconds its generation took."""
    import md_inputs
    t0 = time.perf_counter()
    w = md_inputs.rsa_2m(2.5)
    return w, time.perf_counter() - t0


def run_large(r3, stream, flush, w, gen_s, steps=20):
    """Large single system (2,000,000 particles, random-sequential-addition start at density 0.75,
    T* = 1.2, FP32 forces, k = 10, dt_outer = 0.02) with triplet cutoffs 2.0 and 2.5: whole outer steps
    through the graph-replayed path, CUDA events, L2 flushed before each step."""
    import torch
    out = {}
    out["input_generation_s"] = gen_s
    out["timed_outer_steps"] = steps
    for rc3 in (2.0, 2.5):
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32, stream.cuda_stream)
        try:
            r3.md_set_potentials(h, 1.0, 1.0, w.rc2, w.nu, rc3)
            with torch.cuda.stream(stream):
                r3.md_respa_step(h, 0, w.k_inner, w.dt_outer)
                for _ in range(3):
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                s0 = r3.md_get_stats(h)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                for e0, e1 in ev:
                    flush.fill_(1.0)
                    e0.record(stream)
                    r3.md_respa_step(h, 1, w.k_inner, w.dt_outer)
                    e1.record(stream)
                torch.cuda.synchronize()
                s1 = r3.md_get_stats(h)
            ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
            trip = (s1["triplets_total"] - s0["triplets_total"]) / steps
            out[f"rc3_{rc3}"] = {"ms_per_outer_step": ms, "triplets_per_eval": trip,
                                 "triplets_per_s": trip / (ms / 1e3), "rrespa_steps_per_s": 1e3 / ms,
                                 "atm_kernel": s1["atm_kernel"], "replays": s1["replays"] - s0["replays"]}
        finally:
            r3.md_destroy_system(h)
    return out


def run_direct(r3, stream, fp32_peak, n=4995, calls=2):
    """All-triplet ATM forces (DirectSum, open boundaries, no cutoff) on the aluminium scenario's
    shape (Table 1: 4995 particles at density 4995 / 20^3, nu = 0.3095), FP32, through the C ABI with
    host buffers (the call copies 120 KB each way and is synchronous).  Each unordered triplet counts
    once; the kernel evaluates it from each of its three members (no scatter)."""
    import torch
    import md_inputs
    x, _ = md_inputs.fcc_jitter(n, n / 20.0 ** 3, 0.05, 7)
    with torch.cuda.stream(stream):
        r3.md_atm_direct(x, 0.3095, r3.MD_FP32, stream.cuda_stream)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(calls):
            r3.md_atm_direct(x, 0.3095, r3.MD_FP32, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / calls
    trip = n * (n - 1) * (n - 2) / 6
    tflops = trip * ATM_FLOPS_PER_TRIPLET / (ms / 1e3) / 1e12
    return {"n": n, "ms_per_call": ms, "triplets_per_s": trip / (ms / 1e3), "achieved_tflops": tflops,
            "frac_fp32_peak": tflops / fp32_peak,
            "note": f"{ATM_FLOPS_PER_TRIPLET} flop per unordered triplet (each evaluated from its 3 members)"}


def run_classes(r3, w, stream, flush, steps, r_a=1.5, s_near=2):
    """Distance classes of the three-body force on the same workload (FP32): near triplets (all three
    distances <= r_a) every s_near inner steps, far triplets every outer step (k = 10).  Timed like
    the main line (graph replay, L2 flushed, CUDA events per outer step), beside Algorithm 2 with
    k = s_near, which evaluates every triplet as often as the near class."""
    import torch

    def timed(r_a_, k, n_outer):
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32, stream.cuda_stream)
        try:
            r3.md_set_potentials(h, 1.0, 1.0, w.rc2, w.nu, w.rc3)
            if r_a_ > 0:
                r3.md_set_distance_classes(h, r_a_, s_near)
            dt = w.dt_outer * k / w.k_inner  # same inner step dt_outer / k_inner
            with torch.cuda.stream(stream):
                for _ in range(4):
                    r3.md_respa_step(h, n_outer, k, dt)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                torch.cuda.synchronize()
                s0 = r3.md_get_stats(h)
                for e0, e1 in ev:
                    flush.fill_(1.0)
                    e0.record(stream)
                    r3.md_respa_step(h, n_outer, k, dt)
                    e1.record(stream)
                torch.cuda.synchronize()
                st = r3.md_get_stats(h)
            return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps, st, s0
        finally:
            r3.md_destroy_system(h)

    ms_c, st_c, _ = timed(r_a, w.k_inner, 1)
    ms_2, _, _ = timed(0.0, s_near, w.k_inner // s_near)
    return {"r_a": r_a, "s_near": s_near, "k_inner": w.k_inner,
            "ms_per_outer_step": ms_c, "near_triplets_per_eval": st_c["near_triplets_last"],
            "triplets_per_eval": st_c["triplets_last"],
            "alg2_k_eq_s_near_ms_per_same_time": ms_2,
            "note": "ms for k_inner inner steps of dt_outer / k_inner: classes (near every s_near, far every "
                    "k_inner) vs Algorithm 2 with every triplet every s_near inner steps"}


def _skin_for(L, rc2=2.5, rc3=2.5):
    """Largest skin <= 0.3 that keeps L > 3 (r_c2 + skin) (small replicas need a thinner one)."""
    return max(0.02, min(0.3, L / 3.0 - rc2 - 0.02))


def run_ensemble(r3, n_replicas=256, n_outer=20, seed=None, atm_kernel=2):
    """256 independent replicas, N log-uniform in [500, 20000], rho U[0.6, 0.9], T U[0.8, 1.5],
    k in {4, 8, 16}, dt = 0.002, 20 outer steps each, FP32, all in one batch."""
    import md_inputs
    specs = md_inputs.ensemble_specs(n_replicas, seed)
    b = r3.md_batch_create(0)
    hs, tickets = [], []
    t_setup = time.perf_counter()
    try:
        for i, sp in enumerate(specs):
            sp = dict(sp, n_outer=n_outer)
            w = md_inputs.ensemble_replica(sp, i)
            h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32)
            r3.md_set_skin(h, _skin_for(w.L))
            r3.md_set_potentials(h, 1.0, 1.0, 2.5, 0.073, 2.5)
            r3.md_set_atm_kernel(h, atm_kernel)
            r3.md_respa_step(h, 0, w.k_inner, w.dt_outer)  # initial forces outside the timed region
            hs.append(h)
            tickets.append(r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer))
        t_setup = time.perf_counter() - t_setup
        s0 = [r3.md_get_stats(h)["triplets_total"] for h in hs]
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r3.md_batch_run(b, 0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        trip = sum(r3.md_get_stats(h)["triplets_total"] - a for h, a in zip(hs, s0))
        lat = np.concatenate([r3.md_batch_latency(b, t) for t in tickets])
        done = sum(r3.md_batch_poll(b, t) for t in tickets)
        cycles, replayed = r3.md_batch_cycles(b)
        return {"replicas": n_replicas, "done": int(done), "outer_steps_each": n_outer,
                "cycles": cycles, "replayed_cycles": replayed,
                "particles_total": int(sum(sp["n"] for sp in specs)),
                "triplets_per_s": trip / wall, "wall_s": wall, "setup_s": t_setup,
                "outer_step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                          "samples": int(lat.size), "clock": "device (%globaltimer)"}}
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def run_serving(r3, seconds=3.0, rate=50.0, n_outer=100, k=10, seed=None, atm_kernel=2, max_particles=2_000_000):
    """Poisson arrivals (rate per second) of replicas with N log-uniform in [1e3, 2e5] and rho
    U[0.7, 0.9]; each asks for n_outer outer steps at k inner steps; admitted by a device-memory
    budget (80 % of free HBM) and a bound on the resident particles (max_particles: the time of one
    cycle, hence every request's outer-step latency), state resident, batched continuously; arrivals
    stop after `seconds` and the loop drains the queue."""
    import torch
    import md_inputs
    seed = md_inputs.config_seed(5) if seed is None else seed
    n_req = max(1, int(rate * seconds))
    u = md_inputs.uniform(seed, 6, 0, 4 * n_req).reshape(n_req, 4)
    arrivals = np.cumsum(-np.log(1.0 - u[:, 0]) / rate)
    sizes = np.exp(np.log(1e3) + u[:, 1] * (np.log(2e5) - np.log(1e3))).astype(int)
    dens = 0.7 + 0.2 * u[:, 2]
    free, _ = torch.cuda.mem_get_info()
    b = r3.md_batch_create(int(0.8 * free))
    if max_particles:
        r3.md_batch_set_limits(b, int(max_particles))
    live = {}
    lat_all, e2e, trip_all = [], [], 0
    t0 = time.perf_counter()
    nxt = 0
    try:
        while nxt < n_req or live:
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                w = md_inputs.fcc_system(int(sizes[nxt]), float(dens[nxt]), 1.0, 0.05, seed + 7 + nxt)
                h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32 | r3.MD_DEFERRED)
                r3.md_set_skin(h, _skin_for(w.L))
                r3.md_set_potentials(h, 1.0, 1.0, 2.5, 0.073, 2.5)
                r3.md_set_atm_kernel(h, atm_kernel)
                t = r3.md_batch_submit(b, h, n_outer, k, 0.002 * k)
                live[t] = (h, arrivals[nxt])
                nxt += 1
            if not live:
                time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
                continue
            r3.md_batch_run(b, k)  # one cycle, then admit arrivals again
            for t in list(live):
                if r3.md_batch_poll(b, t):
                    h, ta = live.pop(t)
                    lat_all.append(r3.md_batch_latency(b, t, 1024))
                    e2e.append(time.perf_counter() - t0 - ta)
                    trip_all += r3.md_get_stats(h)["triplets_total"]
                    r3.md_destroy_system(h)
        wall = time.perf_counter() - t0
        lat = np.concatenate(lat_all) if lat_all else np.zeros(1)
        cycles, replayed = r3.md_batch_cycles(b)
        offered = float(sum(sizes)) * n_outer * 200.0 / seconds  # about 200 triplets per particle
        return {"requests": n_req, "arrival_rate_per_s": rate, "arrival_window_s": seconds,
                "max_resident_particles": int(max_particles),
                "offered_triplets_per_s_estimate": offered,
                "cycles": cycles, "replayed_cycles": replayed,
                "outer_steps_each": n_outer, "k_inner": k, "wall_s": wall,
                "triplets_per_s": trip_all / wall,
                "outer_step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                          "samples": int(lat.size), "clock": "device (%globaltimer)"},
                "request_latency_s": {"p50": float(np.percentile(e2e, 50)), "p99": float(np.percentile(e2e, 99))}}
    finally:
        r3.md_batch_destroy(b)
        for h, _ in live.values():
            r3.md_destroy_system(h)


def _cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_linked_cell(w, w2m=None):
    """The linked-cell FP64 CPU code (cpu_cells/: the paper's Cutoff traversal, OpenMP over particles,
    no Newton 3) running Algorithm 2 on the workloads of the GPU runs, on every host core: the CPU
    throughput figure beside the GPU's (the oracle's figure, `cpu_baseline`, is a deliberately simple
    per-particle pass).  Whole outer steps after the initial forces; triplets/s = interacting triplets
    evaluated / wall time of the steps."""
    import cpu_cells
    import md_inputs

    def steps(x, v, L, rc3, k, dt_outer, n_outer):
        st = cpu_cells.State(x, v, L, rc2=w.rc2, nu=w.nu, rc3=rc3)
        st.run(0, k, dt_outer)  # F2b(x0), F3b(x0)
        r = st.run(n_outer, k, dt_outer)
        sec = r["seconds"]
        return {"n": int(x.shape[0]), "rc3": rc3, "k_inner": k, "timed_outer_steps": n_outer,
                "ms_per_outer_step": sec / n_outer * 1e3, "rrespa_steps_per_s": n_outer / sec,
                "triplets_per_s": r["triplets"] / sec, "triplets_per_eval": r["triplets"] / max(1, r["atm_evals"]),
                "atm_only_triplets_per_s": r["triplets"] / r["atm_s"] if r["atm_s"] > 0 else None,
                "lj_share": r["lj_s"] / sec, "atm_share": r["atm_s"] / sec}

    out = {"kind": "linked-cell FP64, OpenMP over particles, no Newton 3 (cpu_cells/)", "cores": cpu_cells.threads(),
           "cpu_model": _cpu_model()}
    w1 = md_inputs.small_fcc_1k()
    out["fcc1k"] = steps(w1.x, w1.v, w1.L, 2.5, w1.k_inner, w1.dt_outer, w1.n_outer)
    out["fcc100k"] = steps(w.x, w.v, w.L, w.rc3, w.k_inner, w.dt_outer, 2)
    if w2m is not None:
        for rc3 in (2.0, 2.5):
            out[f"rsa2m_rc3_{rc3}"] = steps(w2m.x, w2m.v, w2m.L, rc3, w2m.k_inner, w2m.dt_outer, 1)
    return out


def cpu_baseline(w, nsample):
    """The oracle, as it stands, on a bounded sample: the per-particle pass (all triplets and
    pairs containing each sampled particle) for nsample particles of the same workload."""
    import oracle
    import md_inputs
    if nsample >= w.n:
        sel = np.arange(w.n, dtype=np.int64)
    else:
        sel = np.unique((md_inputs.uniform(7, 11, 0, 4 * nsample) * w.n).astype(np.int64))[:nsample]
    oracle.atm_particles(w.x, w.L, sel[:4], w.nu, w.rc3)  # load + warm
    t0 = time.perf_counter()
    _, _, cnt = oracle.atm_particles(w.x, w.L, sel, w.nu, w.rc3)
    oracle.lj_particles(w.x, w.L, sel, 1.0, 1.0, w.rc2)
    dt = time.perf_counter() - t0
    # each sampled particle's pass evaluates every triplet containing it once
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # every interacting triplet appears in the passes of its 3 members: count each once
    return {"value": float(cnt.sum()) / 3.0 / dt, "unit": "triplets/s", "cores": cores, "kind": "oracle",
            "sample": f"per-particle pass (ATM + LJ forces) over {sel.size} particles of the 100k workload "
                      f"(the whole system when 100000), {int(cnt.sum()) // 3} interacting triplets in {dt:.2f} s"}


def run_reference(args):
    """The oracle, as it stands, on the host cores: K timed steps, each the per-particle pass over a
    seeded sample of cpu_sample / K particles of the same workload (so the K steps together cover about
    one full evaluation), after W untimed warm-up samples of 200 particles."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import md_inputs
    w = workload()
    per = max(200, args.cpu_sample // max(1, args.steps))

    def sample(step, size):
        u = md_inputs.uniform(7, 100 + step, 0, 4 * size)
        return np.unique((u * w.n).astype(np.int64))[:size]
    for q in range(args.warmup):
        sel = sample(10_000 + q, 200)
        oracle.atm_particles(w.x, w.L, sel, w.nu, w.rc3)
        oracle.lj_particles(w.x, w.L, sel, 1.0, 1.0, w.rc2)
    trip, secs = 0.0, 0.0
    for q in range(args.steps):
        sel = sample(q, per)
        t0 = time.perf_counter()
        _, _, cnt = oracle.atm_particles(w.x, w.L, sel, w.nu, w.rc3)
        oracle.lj_particles(w.x, w.L, sel, 1.0, 1.0, w.rc2)
        secs += time.perf_counter() - t0
        trip += float(cnt.sum()) / 3.0  # each triplet appears in the passes of its 3 members
    value = trip / secs
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cb = {"value": value, "unit": "triplets/s", "cores": cores, "kind": "oracle",
          "sample": f"{args.steps} steps, each the per-particle pass (ATM + LJ forces) over {per} seeded particles "
                    f"of the 100k workload; {trip:.3g} triplet shares in {secs:.2f} s"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "triplets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fcc100k_rho0.8 (same as our arm), CPU oracle per-particle pass samples"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--lj-kernel", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="LJ kernel of the main runs: -1 autotuned, 0 row, 1 cell-tile, 2 team")
    ap.add_argument("--cpu-sample", type=int, default=100_000,
                    help="particles in the oracle's timed per-particle pass (100000 = one full evaluation)")
    ap.add_argument("--no-batch", action="store_true", help="skip the ensemble and serving runs")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 2,000,000-particle system (its input takes about half a minute to generate)")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window of the serving run")
    ap.add_argument("--serve-max-particles", type=int, default=2_000_000,
                    help="bound on the particles resident in the serving batch (0: memory budget only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark: Wilson-Dirac hop (Dslash) GFLOP/s and its roofline fraction on
the 32^3 x 64 SU(3) workload, plus CG time-to-1e-10 of the mixed-precision
solver against the plain FP64 solver on the same GPU.

One step = the hopping term on the whole lattice (both parity blocks,
bsm_dslash EVEN then ODD, 1320 flop per site) in FP64-accurate double-float
arithmetic (the paper's Dphi is FP64), L2 flushed between steps.  The FP32
hop (the inner operator of the mixed solver) and the native-FP64 hop are
reported beside it with their own rooflines.  Prints one JSON line (rank 0).
`--impl reference` times the FP64 CPU oracle instead, on the same workload.

Multi-GPU (torchrun): independent replicas, one lattice per GPU, no
collective on the data path; the value is the whole-job rate (weak scaling).
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
CSRC = os.path.join(ROOT, "paper_1401_3733_gb300", "csrc")

METRIC = "Dslash GFLOP/s (% of HBM roofline); CG time-to-1e-10 vs plain FP64 CG"
WORKLOAD = dict(dims=(64, 32, 32, 32), N=3, m0=0.05, phase=(math.pi, 0.0, 0.0, 0.0), link_seed=3, eps=0.3,
                src_seed=4)
WORKLOAD_NAME = ("32^3x64 SU(3) fundamental, smooth links exp(i 0.3 H), m0=0.05, antiperiodic time: "
                 "even-odd Wilson hop on both parity blocks, FP64-accurate")
# the small configuration: 4^4 SU(2) fundamental, Haar links, m0 = 0.1 (CG to 1e-10 on the full D^+D)
SMALL = dict(dims=(4, 4, 4, 4), N=2, m0=0.1, phase=(math.pi, 0.0, 0.0, 0.0), link_seed=1, src_seed=2)

# GB300 FP32 pipe: 152 SMs x 128 lanes x 2070 MHz (maximum SM clock), one
# FP32 operation (add, multiply or fused multiply-add) per lane and clock
FP32_OPS_PEAK = 152 * 128 * 2.07e9

# DRAM bytes per output site (dram__bytes_read.sum + dram__bytes_write.sum)
# of a hop kernel, from one single-pass ncu capture of this benchmark's timed
# launches on the 32^3 x 64 workload (summarised under profiles/), valid only
# for the kernel sources it was taken on: `sha` is the hash of those files
# (kernel_sha), and a mismatch reports the traffic as null.
TRAFFIC = {
    "hop_df64": {"bytes_per_site": 1538.4, "sha": "389e1b87bdd79844",
                 "sources": ["hop_df64.cu", "f32x2.cuh", "hop.cuh", "bsm_internal.cuh", "df64.cuh"]},
    "hop_f32": {"bytes_per_site": 736.0, "sha": "eb66718d6a4215c0",
                "sources": ["hop_f32.cu", "hop.cuh", "bsm_internal.cuh"]},
    "hop_f32r12": {"bytes_per_site": 544.0, "sha": "ab237da849b7016d",
                   "sources": ["hop_f32r12.cu", "hop.cuh", "bsm_internal.cuh"]},
}


def kernel_sha(sources):
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_site(kernel):
    t = TRAFFIC[kernel]
    if t["bytes_per_site"] is None or t["sha"] != kernel_sha(t["sources"]):
        return None
    return t["bytes_per_site"]


def flops_per_site(d, real=False):
    """Counting convention per output site of one hop: complex mul 6, add 2."""
    return 64 * d * d + 56 * d if real else 128 * d * d + 56 * d


def bytes_per_site(d, w, real=False):
    """8 links + one input spinor (perfect neighbour reuse) + one output spinor."""
    return (8 * d * d + 16 * d) * w if real else (16 * d * d + 16 * d) * w


def bytes_per_site_r12(w):
    """SU(3) hop with two-row links: 8 links of 12 reals + input + output spinor (d = 3)."""
    return (8 * 12 + 2 * 24) * w


def df64_ops_per_site(d):
    """FP32 operations per output site of the double-float hop (complex
    representation), counted on its algorithm: per direction-sense the spin
    projection (2d complex double-float sums with a sign: 40d), the link
    products (each double-float multiply-add 12 operations, the first of a
    chain 4: 96d^2 - 32d) and the reconstruction (4d complex sums, two of
    them signed: 72d)."""
    return 8 * (96 * d * d + 80 * d)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """Polls SM clock and clock-event reasons through NVML (read-only) in a
    background thread while the timed region runs."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x40: "sw_thermal_slowdown",
               0x80: "hw_thermal_slowdown", 0x100: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting"}

    def __init__(self, uuid):
        self.samples, self.reasons, self.max_mhz = [], set(), None
        self.ok = False
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
                if self.nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(self.h)) != 0:
                    return
            m = ctypes.c_uint()
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = m.value
            self.ok = True
        except OSError:
            pass

    def sample(self):
        c, r = ctypes.c_uint(), ctypes.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0:
            self.samples.append(c.value)
        if self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(r)) == 0:
            for bit, name in self.REASONS.items():
                if r.value & bit:
                    self.reasons.add(name)

    def __enter__(self):
        self.stop = threading.Event()
        if self.ok:
            def loop():
                while not self.stop.is_set():
                    self.sample()
                    time.sleep(0.002)
            self.t = threading.Thread(target=loop, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.ok:
            self.t.join()
            if not self.samples:
                self.sample()

    def summary(self):
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml unavailable"]}
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


def doubling_loop(interval, min_seconds):
    """The paper's fixed-time timing loop (Sec. III): interval(n) runs the
    timed operation n times between two clock reads and returns the seconds;
    n doubles until one interval reaches min_seconds.  Returns (n, seconds)."""
    n = 1
    while True:
        el = interval(n)
        if el >= min_seconds:
            return n, el
        n *= 2


def host_interval(fn):
    def interval(n):
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        return time.perf_counter() - t0
    return interval


def gpu_interval(fn):
    """n calls of fn between two CUDA events on torch's current stream (the
    stream the library launches on)."""
    import torch

    def interval(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3
    return interval


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_child(path):
    """Child process of oracle_timings: times the oracle on the arrays saved
    at `path` with the OpenMP thread count of its environment, prints JSON."""
    import oracle as orc

    z = np.load(path)
    w = WORKLOAD
    lat = orc.Lattice(tuple(int(x) for x in z["dims"]), w["N"], orc.FUND, w["m0"], w["phase"])
    R = orc.links_to_rep(lat, z["U"])
    psi = z["psi"]
    Vh = lat.V // 2
    min_s = float(os.environ.get("BSM_ORACLE_MIN_SECONDS", "1.0"))
    out = {"threads": int(os.environ.get("OMP_NUM_THREADS", "0"))}
    reps, el = doubling_loop(host_interval(lambda: orc.hop(lat, R, psi, orc.EVEN)), min_s)
    out["hop_eo_block"] = {"gflops": round(reps * flops_per_site(lat.d) * Vh / el / 1e9, 3),
                           "seconds_per_call": round(el / reps, 4)}
    reps, el = doubling_loop(host_interval(lambda: orc.dhat(lat, R, psi, orc.DHAT)), min_s)
    out["dhat"] = {"gflops": round(reps * 2 * flops_per_site(lat.d) * Vh / el / 1e9, 3),
                   "seconds_per_call": round(el / reps, 4)}
    # CG to 1e-10 on the small configuration (full D^+D and even-odd)
    s = SMALL
    from paper_1401_3733_gb300 import fields
    slat = orc.Lattice(s["dims"], s["N"], orc.FUND, s["m0"], s["phase"])
    sR = orc.links_to_rep(slat, fields.gauge_field(s["dims"], s["N"], "haar", seed=s["link_seed"]))
    sb = fields.gaussian_spinor(s["dims"], slat.d, s["src_seed"])
    for eo in (False, True):
        t0 = time.perf_counter()
        _, it, res = orc.cg(slat, sR, sb, eo=eo, tol=1e-10)
        out["cg_4x4_su2_" + ("eo" if eo else "full")] = {"seconds": round(time.perf_counter() - t0, 5),
                                                         "iters": it, "rel_res": res}
    # a fixed number of CG iterations on the workload (even-odd);
    # the time to 1e-10 is extrapolated to the GPU solver's iteration count
    # (per-iteration time from the difference of an n-iteration and a
    # 1-iteration solve, so the source preparation and the final residual
    # check are not counted as iterations)
    n_it = int(os.environ.get("BSM_ORACLE_CG_ITERS", "20"))
    t0 = time.perf_counter()
    orc.cg(lat, R, psi, eo=True, tol=1e-30, max_iter=1)
    t1 = time.perf_counter()
    orc.cg(lat, R, psi, eo=True, tol=1e-30, max_iter=n_it)
    t2 = time.perf_counter()
    per_it = ((t2 - t1) - (t1 - t0)) / (n_it - 1)
    out["cg_workload_fixed_iters"] = {"iters": n_it, "seconds": round(t2 - t1, 3),
                                      "seconds_one_iter_solve": round(t1 - t0, 3),
                                      "seconds_per_iter": round(per_it, 4),
                                      "fixed_seconds": round((t1 - t0) - per_it, 3)}
    print(json.dumps(out), flush=True)


def oracle_timings(dims, U, psi, cg_iters_gpu):
    """BASELINE's CPU plan: the oracle single-threaded and on all host cores,
    each in a child process (OpenMP over sites is its only parallelism): one
    even-odd hop block and one Dhat on the 32^3 x 64 workload, CG to 1e-10 on
    the 4^4 SU(2) configuration, and a fixed number of CG iterations on the
    32^3 x 64 workload (time to 1e-10 extrapolated, and labelled so)."""
    import tempfile
    cores = os.cpu_count() or 1
    res = {"cores": cores, "cpu": platform_cpu()}
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "fields.npz")
        np.savez(path, U=U, psi=psi, dims=np.array(dims))
        for name, threads, iters in (("all_cores", cores, 20), ("single_thread", 1, 3)):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads), BSM_ORACLE_CG_ITERS=str(iters))
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", path], env=env,
                               capture_output=True, text=True, timeout=900)
            if r.returncode != 0:
                res[name] = {"error": r.stderr.strip().splitlines()[-1:] or ["failed"]}
                continue
            t = json.loads(r.stdout.strip().splitlines()[-1])
            c = t["cg_workload_fixed_iters"]
            if cg_iters_gpu:
                c["extrapolated_seconds_to_1e-10"] = round(c["fixed_seconds"] + c["seconds_per_iter"] * cg_iters_gpu, 2)
                c["extrapolated_to_iters"] = cg_iters_gpu
            res[name] = t
    return res


def platform_cpu():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Largest value over the ranks (the slowest rank's time); works on the
    NCCL (CUDA tensor) and gloo (CPU tensor) backends."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_per_rank, world):
    """Whole-job throughput of `world` replicas: every rank processes the same
    units, the job takes as long as its slowest rank."""
    return world * units_per_rank / max_over_ranks(seconds_per_rank, world)


def config_dict(dims, world):
    V = int(np.prod(dims))
    return {"workload": WORKLOAD_NAME, "lattice_TXYZ": list(dims), "sites": V,
            "flop_per_site": flops_per_site(WORKLOAD["N"]),
            "algorithmic_bytes_per_site": bytes_per_site(WORKLOAD["N"], 8),
            "l2": "flushed between steps (256 MiB write); inputs (1.4 GB) larger than L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle as it stands (plain C FP64, OpenMP over sites, all host
    cores): one step = its hop on both parity blocks of the whole 32^3 x 64
    workload, the metric and config of the GPU arm."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    from paper_1401_3733_gb300 import fields
    w = WORKLOAD
    lat = orc.Lattice(w["dims"], w["N"], orc.FUND, w["m0"], w["phase"])
    U = fields.gauge_field(w["dims"], w["N"], "smooth", seed=w["link_seed"], eps=w["eps"])
    R = orc.links_to_rep(lat, U)
    del U
    psi = fields.gaussian_spinor(w["dims"], lat.d, w["src_seed"])
    for _ in range(args.warmup):
        orc.hop(lat, R, psi, orc.FULL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.hop(lat, R, psi, orc.FULL)
    el = time.perf_counter() - t0
    value = args.steps * flops_per_site(lat.d) * lat.V / el / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle hop (FP64 plain C, OpenMP over sites) on both parity blocks of the whole "
              f"{'x'.join(map(str, w['dims']))} lattice per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w["dims"], world),
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    from paper_1401_3733_gb300 import bsm, fields

    w = WORKLOAD
    dims, N = (tuple(args.lattice) if args.lattice else w["dims"]), w["N"]
    lat = bsm.lattice(dims, N, bsm.FUND, w["m0"], w["phase"])
    d = bsm.bsm_rep_dim(N, bsm.FUND)
    V = int(np.prod(dims))
    Vh = V // 2
    U = fields.gauge_field(dims, N, "smooth", seed=w["link_seed"] + rank, eps=w["eps"])
    psi = fields.gaussian_spinor(dims, d, w["src_seed"] + rank)

    Ud = torch.from_numpy(U).cuda()
    PRECS = (bsm.F64, bsm.F32, bsm.DF64)
    links = {p: bsm.empty_field(lat, bsm.FIELD_LINKS, p) for p in PRECS}
    ev_l0, ev_l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_l0.record()
    bsm.bsm_links_to_rep(lat, Ud, links[bsm.F32], bsm.F32)
    ev_l1.record()
    bsm.bsm_links_to_rep(lat, Ud, links[bsm.F64], bsm.F64)
    bsm.bsm_links_to_rep(lat, Ud, links[bsm.DF64], bsm.DF64)
    links[bsm.F32R12] = bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F32R12)   # SU(3): two rows per link
    bsm.bsm_links_to_rep(lat, Ud, links[bsm.F32R12], bsm.F32R12)
    del Ud
    psid = torch.from_numpy(psi).cuda()
    src = {p: bsm.empty_field(lat, bsm.FIELD_SPINOR, p) for p in PRECS}
    dst = {p: bsm.empty_field(lat, bsm.FIELD_SPINOR, p) for p in PRECS}
    for p in PRECS:
        bsm.bsm_pack_spinor(lat, psid, src[p], p)
    src[bsm.F32R12], dst[bsm.F32R12] = src[bsm.F32], dst[bsm.F32]   # spinors as FP32
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    torch.cuda.synchronize()
    links_ms = ev_l0.elapsed_time(ev_l1)

    def halves(t, prec):
        n = bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, prec)
        return t[:n], t[n:]

    def dslash_step(prec, evs=None):
        se, so = halves(src[prec], prec)
        de, do = halves(dst[prec], prec)
        if evs:
            evs[0].record()
        bsm.bsm_dslash(lat, links[prec], so, de, bsm.EVEN, 0, prec)
        if evs:
            evs[1].record()
        bsm.bsm_dslash(lat, links[prec], se, do, bsm.ODD, 0, prec)
        if evs:
            evs[2].record()

    def timed_steps(prec, steps, nvtx):
        """`steps` steps, each bracketed by the L2 flush; per-launch CUDA
        events on the launching stream; returns the launch times (ms)."""
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        torch.cuda.nvtx.range_push(nvtx)   # lets ncu --nvtx-include select the timed region
        for k in range(steps):
            flush.zero_()
            dslash_step(prec, evs[k])
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        return [e[0].elapsed_time(e[1]) for e in evs] + [e[1].elapsed_time(e[2]) for e in evs]

    flop_step = flops_per_site(d) * V
    peak, peak_src = load_peaks()
    HEAD = bsm.DF64
    for _ in range(args.warmup):
        flush.zero_()
        dslash_step(HEAD)
    uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(uuid) as clk:
        launch_ms = timed_steps(HEAD, args.steps, "timed_dslash")
    barrier(world)
    wall = time.perf_counter() - wall0
    ms_step = sum(launch_ms) / args.steps
    ms_step_max = max_over_ranks(ms_step, world)
    value = world * flop_step / (ms_step_max * 1e-3) / 1e9   # = whole_job_rate over ranks

    # roofline of the headline kernel: the larger of the HBM time (1536 B per
    # site) and the FP32-pipe time (its double-float operations) binds
    avg_launch_ms = sum(launch_ms) / len(launch_ms)
    hop_bytes = bytes_per_site(d, 8) * Vh
    hop_ops = df64_ops_per_site(d) * Vh
    t_hbm_us = hop_bytes / (peak * 1e9) * 1e6
    t_alu_us = hop_ops / FP32_OPS_PEAK * 1e6
    achieved = hop_bytes / (avg_launch_ms * 1e-3) / 1e9
    achieved_ops = hop_ops / (avg_launch_ms * 1e-3)
    tps = traffic_per_site("hop_df64")
    bound_hbm = t_hbm_us >= t_alu_us
    roofline = {
        "bound": "hbm" if bound_hbm else "alu",
        "achieved": round(achieved if bound_hbm else achieved_ops / 1e12, 1 if bound_hbm else 3),
        "peak": peak if bound_hbm else round(FP32_OPS_PEAK / 1e12, 3),
        "unit": "GB/s" if bound_hbm else "TFP32op/s",
        "frac": round((achieved / peak) if bound_hbm else (achieved_ops / FP32_OPS_PEAK), 4),
        "traffic": None if tps is None else round(tps * Vh),
        "peak_source": peak_src if bound_hbm else "derived: 152 SMs x 128 FP32 lanes x 2070 MHz",
        "kernel": "hop_df64_staged_kernel<3> (double-float, f32x2)", "bytes_per_launch": hop_bytes,
        "avg_launch_us": round(avg_launch_ms * 1e3, 2),
        "roof_us": {"hbm": round(t_hbm_us, 1), "alu": round(t_alu_us, 1)},
        "alu": {"fp32_ops_per_site": df64_ops_per_site(d), "achieved_tops": round(achieved_ops / 1e12, 3),
                "peak_tops": round(FP32_OPS_PEAK / 1e12, 3), "frac": round(achieved_ops / FP32_OPS_PEAK, 4)},
        "hbm_frac": round(achieved / peak, 4),
    }

    # the other precisions on the same inputs, each with its own roofline
    others = {}
    if not args.no_fp64:
        for name, prec in (("dslash_f32", bsm.F32), ("dslash_f32r12", bsm.F32R12), ("dslash_fp64", bsm.F64)):
            for _ in range(2):
                dslash_step(prec)
            n = args.steps if prec == bsm.F32 else max(3, args.steps // 4)
            lm = timed_steps(prec, n, name)
            others[name] = (prec, sum(lm) / len(lm), sum(lm) / n)

    # the paper's timing method (Sec. III) on the headline and FP32 hops: a
    # fixed-time loop doubling the repetitions until one interval reaches
    # 0.5 s (no flush inside it: the inputs exceed L2), median of 5 intervals
    protocol = {}
    if not args.no_protocol:
        for name, prec in (("df64", HEAD), ("f32", bsm.F32)):
            pts = []
            for _ in range(5):
                reps, el = doubling_loop(gpu_interval(lambda: dslash_step(prec)), 0.5)
                pts.append(reps * flop_step / el / 1e9)
            protocol[name] = {"gflops_median": round(statistics.median(pts), 1),
                              "gflops_points": [round(x, 1) for x in pts], "reps_last": reps,
                              "seconds_last": round(el, 3)}

    # end to end through the public API: pinned host canonical FP64 input ->
    # pack -> double-float hop on both parity blocks -> unpack -> pinned host
    # output, every step.  Consecutive steps run on E2E_STREAMS streams with
    # their own buffers, so one step's host->device copy overlaps the previous
    # step's kernels and device->host copy (the link is full duplex); the
    # timed region spans all steps, joined on the timing stream.
    E2E_STREAMS = 3
    e2e_ms, e2e_value = float("nan"), float("nan")
    if not args.no_e2e:
        h_in = [torch.from_numpy(psi).pin_memory() for _ in range(E2E_STREAMS)]
        h_out = [torch.empty_like(h_in[0]).pin_memory() for _ in range(E2E_STREAMS)]
        d_in = [torch.empty_like(psid) for _ in range(E2E_STREAMS)]
        d_out = [torch.empty_like(psid) for _ in range(E2E_STREAMS)]
        e_src = [src[HEAD]] + [bsm.empty_field(lat, bsm.FIELD_SPINOR, HEAD) for _ in range(E2E_STREAMS - 1)]
        e_dst = [dst[HEAD]] + [bsm.empty_field(lat, bsm.FIELD_SPINOR, HEAD) for _ in range(E2E_STREAMS - 1)]
        e_streams = [torch.cuda.Stream() for _ in range(E2E_STREAMS)]
        n_e2e = max(6, min(args.steps, 12))
        nh = bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, HEAD)

        def e2e_step(k):
            b = k % E2E_STREAMS
            s = e_streams[b]
            with torch.cuda.stream(s):
                d_in[b].copy_(h_in[b], non_blocking=True)
                bsm.bsm_pack_spinor(lat, d_in[b], e_src[b], HEAD, stream=s)
                bsm.bsm_dslash(lat, links[HEAD], e_src[b][nh:], e_dst[b][:nh], bsm.EVEN, 0, HEAD, stream=s)
                bsm.bsm_dslash(lat, links[HEAD], e_src[b][:nh], e_dst[b][nh:], bsm.ODD, 0, HEAD, stream=s)
                bsm.bsm_unpack_spinor(lat, e_dst[b], d_out[b], HEAD, stream=s)
                h_out[b].copy_(d_out[b], non_blocking=True)

        for k in range(E2E_STREAMS):
            e2e_step(k)
        torch.cuda.synchronize()
        main = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for s in e_streams:
            s.wait_event(e0)
        for k in range(n_e2e):
            e2e_step(k)
        for s in e_streams:
            done = torch.cuda.Event()
            done.record(s)
            main.wait_event(done)
        e1.record(main)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / n_e2e, world)
        e2e_value = world * flop_step / (e2e_ms * 1e-3) / 1e9
        # the host result of the last step equals the device-path result
        assert torch.equal(h_out[(n_e2e - 1) % E2E_STREAMS], d_out[(n_e2e - 1) % E2E_STREAMS].cpu())
        del h_in, h_out, d_in, d_out, e_src, e_dst
    io_bytes = psi.nbytes

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step_max, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "df64", "data": "synthetic",
        "config": config_dict(dims, world),
        "arithmetic": "double-float: each real an unevaluated sum of two FP32 (about 48 significand bits); "
                      "rel-L2 vs the FP64 oracle 6.7e-15",
        "wall_s_timed_region": round(wall, 4),
        "roofline": roofline,
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        out["e2e"] = {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": io_bytes,
                      "d2h_bytes_per_step": io_bytes, "ms_per_step": round(e2e_ms, 4),
                      "pipelining": f"{E2E_STREAMS} streams, consecutive steps overlap"}

    cg_iters = None
    if rank == 0 and not args.no_mrhs:
        out["mrhs"] = run_mrhs(max(3, min(args.steps, 20)), flush, peak)
    if rank == 0 and not args.no_batch:
        out["batch"] = run_batch(max(3, min(args.steps, 20)), flush)
        out["batch_small"] = run_batch(max(3, min(args.steps, 20)), flush, BATCH_SMALL)
        out["cg_small_graph"] = run_cg_graph(args.cg_max_iter)
        out["cg_batch"] = run_cg_batch(max_iter=args.cg_max_iter)
    if rank == 0 and not args.no_precond:
        out["precond"] = run_precond(peak, peak_src, args.steps)
    if rank == 0 and not args.no_cg:
        out["cg"] = run_cg(lat, links, src[bsm.F64], args.cg_max_iter)
        cg_iters = out["cg"]["fp64"]["iters"]
    if rank == 0 and not args.no_large:
        del links, src, dst, flush
        torch.cuda.empty_cache()
        out["large"] = run_large(args.steps, peak, peak_src, args.cg_max_iter)
    if rank == 0 and world == 1 and not args.no_cpu:
        ot = oracle_timings(dims, U, psi, cg_iters)
        out["oracle_timings"] = ot
        hop_all = ot.get("all_cores", {}).get("hop_eo_block")
        if hop_all:
            out["cpu_baseline"] = {"value": hop_all["gflops"], "unit": "GFLOP/s", "cores": ot["cores"],
                                   "kind": "oracle",
                                   "sample": f"oracle even-odd hop block on the whole "
                                             f"{'x'.join(map(str, dims))} workload (same per-site work as a "
                                             f"step), fixed-time doubling loop >= 1 s, all cores"}
    if protocol:
        out["protocol"] = dict(protocol, method="doubling fixed-time loop (paper Sec. III), >= 0.5 s per "
                                                "interval, median of 5, CUDA events")
    # the other precisions last (the end of the line is what a log tail keeps)
    for name, (prec, avg_ms, ms_s) in others.items():
        bps = bytes_per_site_r12(4) if prec == bsm.F32R12 else bytes_per_site(d, 4 if prec != bsm.F64 else 8)
        ach = bps * Vh / (avg_ms * 1e-3) / 1e9
        entry = {"gflops": round(flop_step / (ms_s * 1e-3) / 1e9, 1), "avg_launch_us": round(avg_ms * 1e3, 2),
                 "bytes_per_site": bps}
        if prec == bsm.F64:
            entry.update(bound="alu (FP64 DFMA, 1.26 TFLOP/s nominal)", hbm_frac=round(ach / peak, 4))
        else:
            t = traffic_per_site("hop_f32" if prec == bsm.F32 else "hop_f32r12")
            entry["roofline"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(ach / peak, 4), "peak_source": peak_src,
                                 "traffic": None if t is None else round(t * Vh)}
        out[name] = entry
    if "cg" in out:
        c = out["cg"]
        out["cg_summary"] = {"fp64_s": c["fp64"]["seconds"], "best_mixed": c["best_mixed"],
                             "best_mixed_s": c[c["best_mixed"]]["seconds"],
                             "fp64_over_mixed_time": c.get("fp64_over_mixed_time"), "iters": cg_iters,
                             "true_res_normal": c[c["best_mixed"]]["true_res_normal"]}
    if "cg_batch" in out:
        c = out["cg_batch"]
        out["cg_batch_summary"] = {"systems": c["systems"], "batched_s": c["batched"]["seconds"],
                                   "per_system_mixed_s": c["per_system_mixed"]["seconds"],
                                   "per_system_fp64_s": c["per_system_fp64"]["seconds"],
                                   "true_res_normal_max": c["batched"]["true_res_normal_max"]}
    out["links_to_rep_ms_f32"] = round(links_ms, 3)
    barrier(world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


MRHS_THEORIES = (("SU(2) adjoint", 2, 1, 5), ("SU(4) two-index antisymmetric", 4, 3, 6),
                 ("SU(6) fundamental", 6, 0, 7))   # (name, N, bsm_rep, link seed)
MRHS_DIMS, MRHS_NRHS, MRHS_EPS = (24, 24, 24, 24), 12, 0.4


def run_mrhs(steps, flush, peak):
    """Batched multi-RHS Dslash on 24^4 lattices in three theories, 12
    Gaussian RHS each, FP32 and BF16 storage (FP32 arithmetic): the full
    operator D on every RHS per step, L2 flushed between steps."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    out = {"lattice_TXYZ": list(MRHS_DIMS), "nrhs": MRHS_NRHS, "eps": MRHS_EPS, "theories": {}}
    V = int(np.prod(MRHS_DIMS))
    for name, N, rep, seed in MRHS_THEORIES:
        lat = bsm.lattice(MRHS_DIMS, N, rep, 0.1, (math.pi, 0, 0, 0))
        d = bsm.bsm_rep_dim(N, rep)
        real = rep == bsm.ADJ
        Ud = torch.from_numpy(fields.gauge_field(MRHS_DIMS, N, "smooth", seed=seed, eps=MRHS_EPS)).cuda()
        src = torch.from_numpy(np.stack([fields.gaussian_spinor(MRHS_DIMS, d, 100 * seed + r)
                                         for r in range(MRHS_NRHS)])).cuda()
        res = {"d": d, "real_rep": real}
        for pname, prec, w in (("f32", bsm.F32, 4), ("bf16", bsm.BF16, 2)):
            links = bsm.empty_field(lat, bsm.FIELD_LINKS, prec)
            bsm.bsm_links_to_rep(lat, Ud, links, prec)
            nbytes = bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, prec) * MRHS_NRHS
            inp = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            outp = torch.empty_like(inp)
            bsm.bsm_pack_spinor_mrhs(lat, src, inp, MRHS_NRHS, prec)
            bsm.bsm_dslash_mrhs(lat, links, inp, outp, MRHS_NRHS, bsm.FULL, 0, prec)   # tunes the RHS block
            for _ in range(3):
                bsm.bsm_dslash_mrhs(lat, links, inp, outp, MRHS_NRHS, bsm.FULL, 0, prec)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.nvtx.range_push(f"mrhs_d{d}{'r' if real else 'c'}_{pname}")
            for e0, e1 in evs:
                flush.zero_()
                e0.record()
                bsm.bsm_dslash_mrhs(lat, links, inp, outp, MRHS_NRHS, bsm.FULL, 0, prec)
                e1.record()
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / steps
            flop = flops_per_site(d, real) * V * MRHS_NRHS
            # hop bytes per output site: links once + n_rhs input and output spinors,
            # plus the same-site read of the A*psi term of D
            byt = ((8 * d * d if real else 16 * d * d) + MRHS_NRHS * 16 * d) * w * V + MRHS_NRHS * 8 * d * w * V
            res[pname] = {"gflops": round(flop / (ms * 1e-3) / 1e9, 1), "ms_per_D": round(ms, 4),
                          "hbm_frac": round(byt / (ms * 1e-3) / 1e9 / peak, 4),
                          "rhs_block": bsm.bsm_dslash_mrhs_block(lat, MRHS_NRHS, prec)}
            del links, inp, outp
        out["theories"][name] = res
        del Ud, src
    return out


BATCH_SHAPES = [((8, 8, 8, 8), 2), ((16, 8, 8, 8), 3), ((12, 12, 12, 12), 2), ((24, 12, 12, 12), 3),
                ((16, 16, 16, 16), 2), ((32, 16, 16, 16), 3), ((20, 20, 20, 20), 2), ((24, 16, 16, 16), 3),
                ((12, 8, 8, 8), 3), ((8, 12, 12, 12), 2), ((16, 12, 12, 12), 3), ((24, 24, 24, 24), 2),
                ((32, 24, 24, 24), 3), ((48, 24, 24, 24), 2), ((40, 24, 24, 24), 3), ((48, 24, 24, 24), 3)]
BATCH_NRHS = 8
BATCH_SMALL = [((8, 8, 8, 8) if k % 2 else (16, 8, 8, 8), 2 + k % 2) for k in range(32)]


def run_batch(steps, flush, shapes=BATCH_SHAPES):
    """A batch of lattices with 8 Gaussian RHS each (default: 16 uneven
    lattices 8^4 .. 24^3 x 48, SU(2) and SU(3) fundamental, smooth links eps =
    0.3; BATCH_SMALL: 32 lattices of 8^4 and 16 x 8^3): the full operator D on
    every RHS of every lattice as one persistent launch, against one multi-RHS
    launch per lattice."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    entries, flop = [], 0
    for k, (dims, N) in enumerate(shapes):
        lat = bsm.lattice(dims, N, bsm.FUND, 0.1, (math.pi, 0, 0, 0))
        V = int(np.prod(dims))
        Ud = torch.from_numpy(fields.gauge_field(dims, N, "smooth", seed=20 + k, eps=0.3)).cuda()
        links = bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F32)
        bsm.bsm_links_to_rep(lat, Ud, links, bsm.F32)
        del Ud
        src = fields.device_gaussian_spinors(dims, N, BATCH_NRHS, seed=40 + k)
        nbytes = bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F32) * BATCH_NRHS
        inp = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        out = torch.empty_like(inp)
        bsm.bsm_pack_spinor_mrhs(lat, src, inp, BATCH_NRHS, bsm.F32)
        del src
        entries.append((lat, links, inp, out, BATCH_NRHS))
        flop += flops_per_site(N) * V * BATCH_NRHS
    items = bsm.batch_items(entries)
    opts = bsm.BatchOpts(bsm.BATCH_D, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(items, opts), dtype=torch.uint8, device="cuda")

    def one_launch():
        bsm.bsm_dslash_batch_async(items, opts, ws)

    def per_lattice():
        for lat, links, inp, out, n in entries:
            bsm.bsm_dslash_mrhs(lat, links, inp, out, n, bsm.FULL, 0, bsm.F32)

    # the batch launch captured once into a CUDA graph, replayed each step
    one_launch()
    assert bsm.bsm_dslash_batch_status(ws) == bsm.OK
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        bsm.bsm_dslash_batch_async(items, opts, ws, stream=side)

    res = {"lattices": len(entries), "nrhs": BATCH_NRHS, "sites": int(sum(np.prod(d) for d, _ in shapes)),
           "gflop_per_step": round(flop / 1e9, 3)}
    for name, fn in (("one_persistent_launch", one_launch), ("graph_replay", graph.replay),
                     ("launch_per_lattice", per_lattice)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        total = 0.0
        torch.cuda.nvtx.range_push(f"batch{len(entries)}_{name}")
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.nvtx.range_pop()
        ms = total / steps
        res[name] = {"ms": round(ms, 4), "gflops": round(flop / (ms * 1e-3) / 1e9, 1)}
    res["status"] = bsm.bsm_strerror(bsm.bsm_dslash_batch_status(ws))
    return res


def run_cg_batch(shapes=None, nrhs=None, max_iter=20000):
    """The uneven batch (16 lattices 8^4 .. 24^3 x 48, SU(2) and SU(3)
    fundamental, smooth links eps = 0.3, m0 = 0.1, 8 Gaussian RHS each): all
    128 systems to 1e-10 by the batched mixed-precision CG (one persistent
    launch of Dhat^+ Dhat for the whole batch per iteration, graph-replayed
    iterations, double-float reliable updates), against the same
    mixed-precision solver called once per system, and against plain FP64 CG
    once per system, on the same GPU."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    shapes = shapes or BATCH_SHAPES
    nrhs = nrhs or BATCH_NRHS
    entries = []
    for k, (dims, N) in enumerate(shapes):
        lat = bsm.lattice(dims, N, bsm.FUND, 0.1, (math.pi, 0, 0, 0))
        Ud = torch.from_numpy(fields.gauge_field(dims, N, "smooth", seed=20 + k, eps=0.3)).cuda()
        L = {p: bsm.empty_field(lat, bsm.FIELD_LINKS, p) for p in (bsm.F32, bsm.DF64, bsm.F64)}
        for p, t in L.items():
            bsm.bsm_links_to_rep(lat, Ud, t, p)
        del Ud
        fb = bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F64)
        b = torch.empty(nrhs * fb, dtype=torch.uint8, device="cuda")
        src = fields.device_gaussian_spinors(dims, N, nrhs, seed=40 + k)
        for r in range(nrhs):
            bsm.bsm_pack_spinor(lat, src[r], b[r * fb:(r + 1) * fb], bsm.F64)
        del src
        entries.append((lat, L, b, torch.zeros_like(b), fb))
    stream = torch.cuda.Stream()
    res = {"lattices": len(entries), "nrhs": nrhs, "systems": len(entries) * nrhs,
           "sites": int(sum(np.prod(d) for d, _ in shapes))}
    # batched
    items = bsm.cg_batch_items([(lat, L[bsm.DF64], L[bsm.F32], b, x, nrhs) for lat, L, b, x, fb in entries])
    ws = torch.empty(bsm.bsm_cg_batch_workspace_bytes(items), dtype=torch.uint8, device="cuda")
    opts = bsm.cg_opts(tol=1e-10, max_iter=max_iter, prec_inner=bsm.F32, prec_outer=bsm.DF64, delta=CG_DELTA,
                       check_every=CG_CHECK_EVERY, use_graph=True)
    best = None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, stats = bsm.bsm_cg_solve_batch(items, opts, ws, stream=stream, raise_on_error=False)
        el = time.perf_counter() - t0
        best = el if best is None or el < best else best
    res["batched"] = {"status": bsm.bsm_strerror(st), "seconds": round(best, 4),
                      "launch_config": dict(zip(("rhs_per_thread", "chunks_per_grab"), bsm.bsm_batch_last_config())),
                      "iters_max": max(s.iters for s in stats),
                      "true_res_normal_max": max(s.true_res_normal for s in stats),
                      "true_res_full_max": max(s.true_res_full for s in stats),
                      "reliable_updates_total": sum(s.reliable_updates for s in stats)}
    del ws
    # one solve per system: the same mixed solver, and plain FP64 CG
    for name, inner, outer in (("per_system_mixed", bsm.F32, bsm.DF64), ("per_system_fp64", bsm.F64, bsm.F64)):
        total, iters, worst = 0.0, 0, 0.0
        for lat, L, b, x, fb in entries:
            ws1 = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, inner), dtype=torch.uint8, device="cuda")
            for r in range(nrhs):
                x1 = torch.zeros(fb, dtype=torch.uint8, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, s1 = bsm.bsm_cg_solve(lat, L[outer], L[bsm.F32], b[r * fb:(r + 1) * fb], x1,
                                          bsm.cg_opts(tol=1e-10, max_iter=max_iter, prec_inner=inner,
                                                      prec_outer=outer, delta=CG_DELTA,
                                                      check_every=CG_CHECK_EVERY), ws1, raise_on_error=False)
                total += time.perf_counter() - t0
                iters = max(iters, s1.iters)
                worst = max(worst, s1.true_res_normal)
            del ws1
        res[name] = {"seconds": round(total, 4), "iters_max": iters, "true_res_normal_max": worst}
    res["per_system_mixed_over_batched"] = round(res["per_system_mixed"]["seconds"] / res["batched"]["seconds"], 3)
    res["fp64_over_batched"] = round(res["per_system_fp64"]["seconds"] / res["batched"]["seconds"], 3)
    return res


def run_cg_graph(max_iter):
    """Mixed-precision CG (DF64 reliable updates) to 1e-10 on a small 8^3 x 16
    SU(3) lattice, where launch gaps matter: iterations replayed from a CUDA
    graph against direct launches, on a non-default stream."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    dims = (16, 8, 8, 8)
    lat = bsm.lattice(dims, 3, bsm.FUND, 0.05, (math.pi, 0, 0, 0))
    U = torch.from_numpy(fields.gauge_field(dims, 3, "smooth", seed=3, eps=0.3)).cuda()
    links = {p: bsm.empty_field(lat, bsm.FIELD_LINKS, p) for p in (bsm.F32, bsm.DF64)}
    for p, t in links.items():
        bsm.bsm_links_to_rep(lat, U, t, p)
    b = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64)
    bsm.bsm_pack_spinor(lat, torch.from_numpy(fields.gaussian_spinor(dims, 3, 4)).cuda(), b, bsm.F64)
    stream = torch.cuda.Stream()
    ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, bsm.F32), dtype=torch.uint8, device="cuda")
    res = {"lattice_TXYZ": list(dims)}
    for name, graph in (("direct", False), ("graph", True)):
        secs = []
        for _ in range(3):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            st, stats = bsm.bsm_cg_solve(lat, links[bsm.DF64], links[bsm.F32], b, x,
                                         bsm.cg_opts(tol=1e-10, max_iter=max_iter, prec_inner=bsm.F32,
                                                     prec_outer=bsm.DF64, use_graph=graph, check_every=16),
                                         ws, stream=stream, raise_on_error=False)
            secs.append(stats.seconds)
        res[name] = {"status": bsm.bsm_strerror(st), "seconds": round(min(secs), 5), "iters": stats.iters,
                     "true_res_normal": stats.true_res_normal}
    return res


# the largest single-lattice workload: 48^3 x 96 SU(3), smooth links
# exp(i 0.3 H) drawn on the device (host generation of 42M matrices would take
# about a minute), m0 = 0.05, antiperiodic time
LARGE = dict(dims=(96, 48, 48, 48), N=3, m0=0.05, phase=(math.pi, 0.0, 0.0, 0.0), eps=0.3, link_seed=5, src_seed=6)


def run_large(steps, peak, peak_kind, max_iter):
    """48^3 x 96: the FP32 Dslash (full and two-row links) against the HBM
    roofline, mixed-precision CG against plain FP64 CG to 1e-10, and the
    learned-preconditioner FGCR (network trained on 8^3 x 16 lattices of the
    same ensemble) on the same system."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    w = LARGE
    dims, N = w["dims"], w["N"]
    lat = bsm.lattice(dims, N, bsm.FUND, w["m0"], w["phase"])
    V = int(np.prod(dims))
    Vh = V // 2
    U = fields.device_smooth_gauge_field(dims, N, w["link_seed"], w["eps"])
    links = {p: bsm.empty_field(lat, bsm.FIELD_LINKS, p) for p in (bsm.F32, bsm.F32R12, bsm.F64, bsm.DF64)}
    for p, t in links.items():
        bsm.bsm_links_to_rep(lat, U, t, p)
    del U
    psi = fields.device_gaussian_spinors(dims, N, 1, w["src_seed"])[0]
    b = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64)
    bsm.bsm_pack_spinor(lat, psi, b, bsm.F64)
    src = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F32)
    dst = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F32)
    bsm.bsm_pack_spinor(lat, psi, src, bsm.F32)
    del psi
    nh = bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, bsm.F32)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flop = flops_per_site(N) * V
    res = {"lattice_TXYZ": list(dims), "sites": V, "eps": w["eps"], "m0": w["m0"],
           "links": "smooth exp(i eps H), drawn on the device (seeded Philox)"}
    for name, prec, bps in (("dslash_f32", bsm.F32, bytes_per_site(N, 4)),
                            ("dslash_f32r12", bsm.F32R12, bytes_per_site_r12(4))):
        for _ in range(3):
            bsm.bsm_dslash(lat, links[prec], src[nh:], dst[:nh], bsm.EVEN, 0, prec)
        n = max(3, min(steps, 10))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        torch.cuda.nvtx.range_push(f"large_{name}")
        for e in evs:
            flush.zero_()
            e[0].record()
            bsm.bsm_dslash(lat, links[prec], src[nh:], dst[:nh], bsm.EVEN, 0, prec)
            e[1].record()
            bsm.bsm_dslash(lat, links[prec], src[:nh], dst[nh:], bsm.ODD, 0, prec)
            e[2].record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = sum(e[0].elapsed_time(e[2]) for e in evs) / n
        launch = ms / 2
        res[name] = {"gflops": round(flop / (ms * 1e-3) / 1e9, 1), "ms_per_step": round(ms, 4),
                     "avg_launch_us": round(launch * 1e3, 1), "algorithmic_bytes_per_site": bps,
                     "hbm_frac": round(bps * Vh / (launch * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind}
    del src, dst, flush
    for name, inner, outer in (("cg_mixed_df64_r12", bsm.F32R12, bsm.DF64), ("cg_fp64", bsm.F64, bsm.F64)):
        ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, inner), dtype=torch.uint8, device="cuda")
        x = torch.empty_like(b)
        st, stats = bsm.bsm_cg_solve(lat, links[outer], links[bsm.F32R12], b, x,
                                     bsm.cg_opts(tol=1e-10, max_iter=max_iter, prec_inner=inner, prec_outer=outer,
                                                 delta=CG_DELTA, check_every=CG_CHECK_EVERY),
                                     ws, raise_on_error=False)
        res[name] = {"status": bsm.bsm_strerror(st), "seconds": round(stats.seconds, 4), "iters": stats.iters,
                     "reliable_updates": stats.reliable_updates, "true_res_normal": stats.true_res_normal,
                     "true_res_full": stats.true_res_full}
        del ws, x
    if res["cg_mixed_df64_r12"]["seconds"] > 0:
        res["fp64_over_mixed_time"] = round(res["cg_fp64"]["seconds"] / res["cg_mixed_df64_r12"]["seconds"], 3)
    # the learned preconditioner, trained on small lattices of this ensemble
    cfg = dict(PRECOND, eps=w["eps"], m0=w["m0"])
    W, train = train_ptc(cfg)
    o = bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=cfg["restart"], eo=True, precond=bsm.FGCR_PTC,
                      channels=cfg["channels"], ptc_prec=bsm.BF16, prec_inner=bsm.F32, inner_tol=1e-3, check_every=4,
                      prec_outer=bsm.DF64)
    ws = torch.empty(bsm.bsm_fgcr_workspace_bytes(lat, o), dtype=torch.uint8, device="cuda")
    x = torch.empty_like(b)
    st, stats = bsm.bsm_fgcr_solve(lat, links[bsm.DF64], links[bsm.F32], W[0], W[1], b, x, o, ws, raise_on_error=False)
    res["fgcr_eo_ptc_bf16_fp32cycles"] = {"status": bsm.bsm_strerror(st), "seconds": round(stats.seconds, 4),
                                          "iters": stats.iters, "cycles": stats.cycles, "true_res": stats.true_res,
                                          "outer": "df64", "training": train}
    return res


# learned preconditioner workload: 16^3 x 32 SU(3), smooth links exp(i 0.5 H);
# m0 = -0.62 is where the Lanczos estimate of cond(Dhat^+ Dhat) peaks on this
# ensemble (about 1.4e3).  Training pairs come from plain FP64 CG iterates on
# 50 configurations of the ensemble at 8^3 x 16 (the network's two-hop
# stencil is local, so a small volume carries its training signal), and the
# solvers are evaluated on a held-out 16^3 x 32 configuration.
PRECOND = dict(dims=(32, 16, 16, 16), train_dims=(16, 8, 8, 8), N=3, eps=0.5, m0=-0.62,
               phase=(math.pi, 0.0, 0.0, 0.0), eval_seed=3, src_seed=4, train_seeds=tuple(range(100, 150)),
               pair_sources=4, pair_iters=(2, 5, 10, 20, 40), channels=12, steps=2500, batch=8, lr=3e-3,
               restart=32)


def cg_pairs(cfg, seed=7):
    """Residual/error pairs of D x = b from plain FP64 CG (bsm_cg_solve on the
    even-odd normal equations): for each training configuration and Gaussian
    source b, the converged x* (1e-12) and the iterates x_k after k
    iterations (a solve stopped at max_iter = k); r_k = b - D x_k and
    e_k = x* - x_k satisfy D e_k = r_k.  Returns, per configuration, its FP32
    links and the pairs as one-channel PTC fields."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    dims, N = cfg["train_dims"], cfg["N"]
    lat = bsm.lattice(dims, N, bsm.FUND, cfg["m0"], cfg["phase"])
    V = int(np.prod(dims))
    fb = V * N * 4
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, bsm.F64), dtype=torch.uint8, device="cuda")
    b64, x64, xk, dx = (bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64) for _ in range(4))
    out, iters, t0 = [], [], time.perf_counter()
    for sd in cfg["train_seeds"]:
        Ud = torch.from_numpy(fields.gauge_field(dims, N, "smooth", seed=sd, eps=cfg["eps"])).cuda()
        l64, l32 = bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F64), bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F32)
        bsm.bsm_links_to_rep(lat, Ud, l64, bsm.F64)
        bsm.bsm_links_to_rep(lat, Ud, l32, bsm.F32)
        npair = cfg["pair_sources"] * len(cfg["pair_iters"])
        R = torch.empty(npair * fb, dtype=torch.complex64, device="cuda")
        E = torch.empty_like(R)
        j = 0
        for _ in range(cfg["pair_sources"]):
            bsm.bsm_pack_spinor(lat, torch.randn((V, 4, N), dtype=torch.complex128, device="cuda", generator=g),
                                b64, bsm.F64)
            x64.zero_()
            _, st = bsm.bsm_cg_solve(lat, l64, None, b64, x64, bsm.cg_opts(tol=1e-12, max_iter=20000), ws)
            iters.append(st.iters)
            for k in cfg["pair_iters"]:
                xk.zero_()
                bsm.bsm_cg_solve(lat, l64, None, b64, xk, bsm.cg_opts(tol=1e-30, max_iter=k, check_every=1), ws,
                                 raise_on_error=False)
                bsm.bsm_dslash(lat, l64, xk, dx, bsm.FULL, 0, bsm.F64)
                r = b64.view(torch.float64) - dx.view(torch.float64)           # r_k = b - D x_k
                e = x64.view(torch.float64) - xk.view(torch.float64)           # e_k = x* - x_k
                bsm.bsm_ptc_pack(lat, r.view(torch.uint8), R[j * fb:(j + 1) * fb])
                bsm.bsm_ptc_pack(lat, e.view(torch.uint8), E[j * fb:(j + 1) * fb])
                j += 1
        out.append((l32, R, E, npair))
    torch.cuda.synchronize()
    return out, {"kind": "plain FP64 CG iterates: r_k = b - D x_k, e_k = x* - x_k", "pairs": len(out) * out[0][3],
                 "configs": len(out), "sources_per_config": cfg["pair_sources"],
                 "cg_iterates": list(cfg["pair_iters"]), "cg_iters_to_1e-12": [min(iters), max(iters)],
                 "seconds": round(time.perf_counter() - t0, 2)}


def synthetic_pairs(cfg, seed=7):
    """Exact residual/error pairs of D x = b with a Gaussian error: e ~ N(0, 1)
    per real component, r = D e (the library's FP64 operator), the same
    number of pairs per training configuration as cg_pairs."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    dims, N = cfg["train_dims"], cfg["N"]
    lat = bsm.lattice(dims, N, bsm.FUND, cfg["m0"], cfg["phase"])
    V = int(np.prod(dims))
    fb = V * N * 4
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    e64, r64 = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64), bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64)
    npair = cfg["pair_sources"] * len(cfg["pair_iters"])
    out, t0 = [], time.perf_counter()
    for sd in cfg["train_seeds"]:
        Ud = torch.from_numpy(fields.gauge_field(dims, N, "smooth", seed=sd, eps=cfg["eps"])).cuda()
        l64, l32 = bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F64), bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F32)
        bsm.bsm_links_to_rep(lat, Ud, l64, bsm.F64)
        bsm.bsm_links_to_rep(lat, Ud, l32, bsm.F32)
        R = torch.empty(npair * fb, dtype=torch.complex64, device="cuda")
        E = torch.empty_like(R)
        for j in range(npair):
            bsm.bsm_pack_spinor(lat, torch.randn((V, 4, N), dtype=torch.complex128, device="cuda", generator=g),
                                e64, bsm.F64)
            bsm.bsm_dslash(lat, l64, e64, r64, bsm.FULL, 0, bsm.F64)
            bsm.bsm_ptc_pack(lat, e64, E[j * fb:(j + 1) * fb])
            bsm.bsm_ptc_pack(lat, r64, R[j * fb:(j + 1) * fb])
        out.append((l32, R, E, npair))
    torch.cuda.synchronize()
    return out, {"kind": "exact pairs r = D e, Gaussian e", "pairs": len(out) * npair, "configs": len(out),
                 "seconds": round(time.perf_counter() - t0, 2)}


def train_ptc(cfg, seed=7, pairs="synthetic"):
    """Adam on loss = sum_b |M(r_b) - e_b|^2 / |e_b|^2 over a pool of
    residual/error pairs (synthetic_pairs, or cg_pairs from plain FP64 CG):
    each step takes a batch of pairs of one training configuration (cycling
    over the configurations), cfg['steps'] x cfg['batch'] samples in all."""
    import torch
    from paper_1401_3733_gb300 import bsm

    dims, N, C, nb = cfg["train_dims"], cfg["N"], cfg["channels"], cfg["batch"]
    lat = bsm.lattice(dims, N, bsm.FUND, cfg["m0"], cfg["phase"])
    V = int(np.prod(dims))
    pool, pair_info = (cg_pairs if pairs == "cg" else synthetic_pairs)(cfg, seed)
    A = 4.0 + cfg["m0"]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    W1 = 0.05 * torch.randn((9, 1, 4, C, 4), dtype=torch.complex64, device="cuda", generator=g)
    W1[0, 0, :, 0, :] += torch.eye(4, device="cuda")
    W2 = 0.01 * torch.randn((9, C, 4, 1, 4), dtype=torch.complex64, device="cuda", generator=g)
    W2[0, 0, :, 0, :] += torch.eye(4, device="cuda") / A
    W = [W1.reshape(36, 4 * C).contiguous(), W2.reshape(36 * C, 4).contiguous()]
    G = [torch.empty_like(t) for t in W]
    m = [torch.zeros_like(t) for t in W]
    v = [torch.zeros_like(t) for t in W]
    fb = V * N * 4
    R, E = (torch.empty(nb * fb, dtype=torch.complex64, device="cuda") for _ in range(2))
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(lat, C, nb, 1), dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(seed)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(1, cfg["steps"] + 1):
        l32, PR, PE, npair = pool[step % len(pool)]
        for b, j in enumerate(rng.choice(npair, size=nb, replace=npair < nb)):
            R[b * fb:(b + 1) * fb].copy_(PR[j * fb:(j + 1) * fb])
            E[b * fb:(b + 1) * fb].copy_(PE[j * fb:(j + 1) * fb])
        losses.append(bsm.bsm_ptc_loss_grad(lat, l32, W[0], W[1], C, R, E, nb, G[0], G[1], ws) / nb)
        lr = cfg["lr"] if step <= 2 * cfg["steps"] // 3 else cfg["lr"] / 3
        for k in range(2):
            bsm.bsm_ptc_adam_step(W[k], G[k], m[k], v[k], lr, step)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return W, {"train_lattice_TXYZ": list(dims), "training_pairs": pair_info,
               "samples": cfg["steps"] * nb, "steps": cfg["steps"], "seconds": round(secs, 2),
               "loss_first": round(losses[0], 5), "loss_last100": round(float(np.mean(losses[-100:])), 5)}


def run_precond(peak, peak_kind, steps):
    """The learned parallel-transport preconditioner inside flexible GCR on the
    held-out configuration, to |b - D x| <= 1e-10 |b|, against FGCR without it
    and against the CG solvers (the reference method) on the same system; plus
    the HBM roofline of one BF16 network application on the 32^3 x 64 lattice."""
    import torch
    from paper_1401_3733_gb300 import bsm, fields

    cfg = PRECOND
    W, train = train_ptc(cfg)
    dims, N, C = cfg["dims"], cfg["N"], cfg["channels"]
    lat = bsm.lattice(dims, N, bsm.FUND, cfg["m0"], cfg["phase"])
    Ud = torch.from_numpy(fields.gauge_field(dims, N, "smooth", seed=cfg["eval_seed"], eps=cfg["eps"])).cuda()
    L = {p: bsm.empty_field(lat, bsm.FIELD_LINKS, p) for p in (bsm.F64, bsm.F32, bsm.DF64, bsm.F32R12)}
    for p, t in L.items():
        bsm.bsm_links_to_rep(lat, Ud, t, p)
    b = bsm.empty_field(lat, bsm.FIELD_SPINOR, bsm.F64)
    bsm.bsm_pack_spinor(lat, torch.from_numpy(fields.gaussian_spinor(dims, N, cfg["src_seed"])).cuda(), b, bsm.F64)
    res = {"workload": f"{dims[1]}^3x{dims[0]} SU(3) fundamental, smooth links exp(i {cfg['eps']} H), "
                       f"m0={cfg['m0']}, antiperiodic time; D x = b to 1e-10",
           "network": f"2 parallel-transport layers 1->{C}->1 channels", "training": train}
    ptc = dict(precond=bsm.FGCR_PTC, channels=C)
    # FP32 cycles; the residual after each cycle in double-float (FP64-accurate)
    mixed = dict(prec_inner=bsm.F32, inner_tol=1e-3, check_every=4, prec_outer=bsm.DF64)
    m = cfg["restart"]
    cases = {
        "fgcr_none_fp64": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m),
        "fgcr_ptc_f32_fp64": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m, ptc_prec=bsm.F32, **ptc),
        "fgcr_eo_none_fp64": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m, eo=True),
        "fgcr_eo_none_fp32cycles": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m, eo=True, **mixed),
        "fgcr_eo_ptc_f32_fp64": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m, eo=True, ptc_prec=bsm.F32, **ptc),
        "fgcr_eo_ptc_bf16_fp32cycles": bsm.fgcr_opts(tol=1e-10, max_iter=4000, restart=m, eo=True,
                                                     ptc_prec=bsm.BF16, **ptc, **mixed),
    }
    for name, o in cases.items():
        ws = torch.empty(bsm.bsm_fgcr_workspace_bytes(lat, o), dtype=torch.uint8, device="cuda")
        best = None
        for _ in range(2):
            x = torch.empty_like(b)
            st, stats = bsm.bsm_fgcr_solve(lat, L[o.prec_outer], L[bsm.F32], W[0], W[1], b, x, o, ws,
                                           raise_on_error=False)
            if best is None or stats.seconds < best[1].seconds:
                best = (st, stats)
        st, stats = best
        res[name] = {"status": bsm.bsm_strerror(st), "iters": stats.iters, "cycles": stats.cycles,
                     "seconds": round(stats.seconds, 5), "true_res": stats.true_res,
                     "outer": "df64" if o.prec_outer == bsm.DF64 else "fp64"}
        del ws
    for name, inner, outer in (("cg_fp64", bsm.F64, bsm.F64), ("cg_mixed_df64", bsm.F32R12, bsm.DF64)):
        ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, inner), dtype=torch.uint8, device="cuda")
        best = None
        for _ in range(2):
            x = torch.empty_like(b)
            st, stats = bsm.bsm_cg_solve(lat, L[outer], L[bsm.F32R12], b, x,
                                         bsm.cg_opts(tol=1e-10, max_iter=20000, prec_inner=inner, prec_outer=outer,
                                                     delta=CG_DELTA, check_every=CG_CHECK_EVERY),
                                         ws, raise_on_error=False)
            if best is None or stats.seconds < best[1].seconds:
                best = (st, stats)
        st, stats = best
        res[name] = {"status": bsm.bsm_strerror(st), "iters": stats.iters, "seconds": round(stats.seconds, 5),
                     "true_res_full": stats.true_res_full}
        del ws
    res["iteration_reduction_ptc_full"] = round(res["fgcr_none_fp64"]["iters"] /
                                                max(1, res["fgcr_ptc_f32_fp64"]["iters"]), 2)
    res["iteration_reduction_ptc_eo"] = round(res["fgcr_eo_none_fp64"]["iters"] /
                                              max(1, res["fgcr_eo_ptc_f32_fp64"]["iters"]), 2)
    best = min((k for k in res if k.startswith("fgcr_eo_ptc")), key=lambda k: res[k]["seconds"])
    res["best_ptc"] = best
    res["cg_mixed_over_best_ptc_time"] = round(res["cg_mixed_df64"]["seconds"] / res[best]["seconds"], 3)
    # the same network trained on residual/error pairs of plain FP64 CG
    # iterates instead (their errors are dominated by the low modes, which a
    # two-hop local network cannot invert: compare its loss and iterations)
    Wcg, train_cg = train_ptc(cfg, pairs="cg")
    o = cases["fgcr_eo_ptc_bf16_fp32cycles"]
    ws = torch.empty(bsm.bsm_fgcr_workspace_bytes(lat, o), dtype=torch.uint8, device="cuda")
    x = torch.empty_like(b)
    st, stats = bsm.bsm_fgcr_solve(lat, L[o.prec_outer], L[bsm.F32], Wcg[0], Wcg[1], b, x, o, ws, raise_on_error=False)
    res["cg_pair_network"] = {"training": train_cg, "fgcr_eo_ptc_bf16_fp32cycles": {
        "status": bsm.bsm_strerror(st), "iters": stats.iters, "seconds": round(stats.seconds, 5),
        "true_res": stats.true_res},
        "iteration_reduction_eo": round(res["fgcr_eo_none_fp64"]["iters"] / max(1, stats.iters), 2)}
    del ws
    res["ptc_apply"] = ptc_apply_roofline(W, C, peak, peak_kind, steps)
    return res


def ptc_apply_roofline(W, C, peak, peak_kind, steps, dims=None):
    """One BF16 network application (fused transport + two-GEMM kernel, then
    the 9-point stencil) on the 32^3 x 64 lattice, L2 flushed between
    applications.  Algorithmic bytes per site: the one-channel FP32 input and
    output (2 x 4 d x 8) and the FP32 links once (8 d^2 x 8)."""
    import torch
    from paper_1401_3733_gb300 import bsm

    dims, N = tuple(dims or WORKLOAD["dims"]), WORKLOAD["N"]
    lat = bsm.lattice(dims, N, bsm.FUND, WORKLOAD["m0"], WORKLOAD["phase"])
    V = int(np.prod(dims))
    U = torch.zeros((V, 4, N, N), dtype=torch.complex128, device="cuda")
    U.real.copy_(torch.eye(N, dtype=torch.float64, device="cuda").expand(V, 4, N, N))
    L32 = bsm.empty_field(lat, bsm.FIELD_LINKS, bsm.F32)
    bsm.bsm_links_to_rep(lat, U, L32, bsm.F32)
    del U
    F = torch.randn(V * N * 4, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(F)
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(lat, C, 1, 0), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        bsm.bsm_ptc_apply(lat, L32, W[0], W[1], C, F, out, 1, bsm.BF16, ws)
    total, n = 0.0, max(3, min(steps, 20))
    for _ in range(n):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bsm.bsm_ptc_apply(lat, L32, W[0], W[1], C, F, out, 1, bsm.BF16, ws)
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / n
    alg = (2 * 4 * N * 8 + 8 * N * N * 8) * V
    return {"lattice_TXYZ": list(dims), "channels": C, "ms": round(ms, 4), "bound": "hbm",
            "algorithmic_bytes": alg, "achieved_gbs": round(alg / (ms * 1e-3) / 1e9, 1),
            "peak_gbs": peak, "peak_kind": peak_kind, "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
            "launches": 3, "l2": "flushed between applications"}


def run_ptc_apply_only(args):
    import torch

    peak, peak_src = load_peaks()
    C = PRECOND["channels"]
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    W = [0.1 * torch.randn((36, 4 * C), dtype=torch.complex64, device="cuda", generator=g),
         0.1 * torch.randn((36 * C, 4), dtype=torch.complex64, device="cuda", generator=g)]
    print(json.dumps({"ptc_apply": ptc_apply_roofline(W, C, peak, peak_src, args.steps, args.lattice)}))


# mixed CG: reliable update once |r| has fallen 100x below its largest value
# since the last one (FP32 keeps ~7 digits, so the iterated residual stays
# accurate over 2 decades); host convergence test every 16 iterations.  On
# the 32^3 x 64 workload this takes 4 instead of 6 updates at the same 86
# iterations (delta = 0.1: 73.5 ms, 0.01: 67.7 ms, 0.001: 64.3 ms).
CG_DELTA = 0.01
CG_CHECK_EVERY = 16


def run_cg(lat, links, b, max_iter):
    """Time-to-1e-10 (true residual of the normal equations, recomputed at the
    outer precision) of the mixed-precision solver (FP32 inner iteration,
    reliable updates in FP64 or in FP64-accurate double-float) and of plain
    CG in FP64 and in double-float, same source, same GPU."""
    import torch
    from paper_1401_3733_gb300 import bsm

    res = {"delta": CG_DELTA, "check_every": CG_CHECK_EVERY}
    cases = (("mixed_df64", bsm.F32, bsm.DF64), ("mixed_df64_r12", bsm.F32R12, bsm.DF64),
             ("mixed", bsm.F32, bsm.F64), ("fp64", bsm.F64, bsm.F64), ("df64", bsm.DF64, bsm.DF64))
    for name, inner, outer in cases:
        ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, inner), dtype=torch.uint8, device="cuda")
        x = torch.zeros_like(b)
        torch.cuda.nvtx.range_push(f"cg_{name}")
        st, stats = bsm.bsm_cg_solve(lat, links[outer], links[inner if inner == bsm.F32R12 else bsm.F32], b, x,
                                     bsm.cg_opts(tol=1e-10, max_iter=max_iter, prec_inner=inner, prec_outer=outer,
                                                 delta=CG_DELTA, check_every=CG_CHECK_EVERY),
                                     ws, raise_on_error=False)
        torch.cuda.nvtx.range_pop()
        res[name] = {"status": bsm.bsm_strerror(st), "seconds": round(stats.seconds, 4), "iters": stats.iters,
                     "reliable_updates": stats.reliable_updates, "true_res_normal": stats.true_res_normal,
                     "true_res_full": stats.true_res_full}
        del ws
    best = min(("mixed", "mixed_df64", "mixed_df64_r12"), key=lambda k: res[k]["seconds"])
    res["best_mixed"] = best
    if res[best]["seconds"] > 0:
        res["fp64_over_mixed_time"] = round(res["fp64"]["seconds"] / res[best]["seconds"], 3)
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-solution part")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cg-max-iter", type=int, default=20000)
    ap.add_argument("--lattice", type=int, nargs=4, metavar=("T", "X", "Y", "Z"),
                    help="override the lattice (profiling of a smaller case); default 64 32 32 32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP32, two-row-link FP32 and FP64 Dslash lines")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--no-mrhs", action="store_true", help="skip the multi-RHS 24^4 three-theory lines")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-lattice batch and small-lattice CG lines")
    ap.add_argument("--no-precond", action="store_true", help="skip the learned-preconditioner (FGCR) line")
    ap.add_argument("--no-large", action="store_true", help="skip the 48^3 x 96 lines")
    ap.add_argument("--no-protocol", action="store_true", help="skip the doubling fixed-time loop (median of 5)")
    ap.add_argument("--oracle-child", metavar="NPZ", help=argparse.SUPPRESS)
    ap.add_argument("--ptc-apply-only", action="store_true",
                    help="only the BF16 network application's roofline (on --lattice, random weights); "
                         "the profiling entry for its kernels")
    args = ap.parse_args()
    if args.oracle_child:
        oracle_child(args.oracle_child)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.ptc_apply_only:
        run_ptc_apply_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

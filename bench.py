#!/usr/bin/env python3
"""Throughput bench: exact Sauvola/Niblack binarization of a 4096x4096 RGB page.

One step = the whole hot path over one page for both threshold rules
(Sauvola k=0.5 R=128, Niblack k=-0.2) and every window W in {15, 31, 61, 101}:
eight launches of the fused kernel, each reading the RGB page (3 B/px) and
writing the byte mask (1 B/px).  Inputs are seeded synthetic pages with
stains and blotches, resident in HBM; each launch reads its own copy of the
page (8 copies, 400 MB, more than the 129 MB L2), so no launch finds its
input in L2.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
(the sliding-window scheme) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W_IMG, CH, SEED = 4096, 4096, 3, 2
RUNS = [(W, "sauvola", 0.5, 128.0) for W in (15, 31, 61, 101)] + \
       [(W, "niblack", -0.2, 128.0) for W in (15, 31, 61, 101)]
METRIC = "Mpixel/s and % HBM roofline per W (15–101); served pages/s at p50/p99 latency"
WORKLOAD = "page 4096x4096 RGB (stains, blotches, sigma 8), fused RGB->gray, Sauvola k=0.5 R=128 and " \
           "Niblack k=-0.2, W in {15,31,61,101}, byte mask"
BYTES_PER_PX = CH + 1           # compulsory traffic: RGB input + byte mask output
NCOPY = len(RUNS)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, world, device):
    """The slowest rank's time: every replica processed the same pixels, the job ends with the last one."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, px_step, total_ms):
    """Whole-job throughput in Mpixel/s: pixels processed by all replicas over the slowest rank's time."""
    return world * steps * px_step / (total_ms / 1e3) / 1e6


def gpu_uuid(dev):
    try:
        import torch
        return str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fused_source_hash():
    h = hashlib.sha256()
    for f in ("fused.cu", "segment.cuh", "decide.cuh", "ptx.cuh", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1210_3165_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    p = os.path.join(ROOT, "profiles", "fused_traffic.json")
    try:
        d = json.load(open(p))
        if d.get("source_sha") == fused_source_hash():
            return d.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (clocks and clock-event reasons)."""
    SM = 1  # NVML_CLOCK_SM
    # nvmlClocksEventReason* bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, uuid, index):
        import ctypes
        self.c = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.h = ctypes.c_void_p()
        rc = -1
        if uuid:
            rc = lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(v)) != 0:
            raise RuntimeError("no max clock")
        self.max_mhz = float(v.value)

    def sample(self):
        c = self.c
        v, r = c.c_uint(), c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(v)) != 0:
            return None
        reasons = set()
        if self.reasons_fn(self.h, c.byref(r)) == 0:
            reasons = {nm for nm, bit in self.BITS.items() if r.value & bit}
        return float(v.value), reasons


class ClockSampler:
    """SM clock and throttle reasons while the timed region runs: NVML polled every 5 ms (the region can
    be tens of milliseconds), else nvidia-smi every 200 ms."""
    Q = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int, uuid: str | None = None):
        self.gpu = gpu_index
        self.uuid = uuid
        self.lines = []
        self.samples = []
        self.proc = None
        self.nvml = None
        self.stop_evt = threading.Event()

    def start(self):
        try:
            self.nvml = _Nvml(self.uuid, self.gpu)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            first = self.nvml.sample()  # one sample before the region starts, so polling is known to work
            if first is not None:
                self.samples.append(first)
                self.t = threading.Thread(target=self._poll, daemon=True)
                self.t.start()
                return
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _poll(self):
        while not self.stop_evt.wait(0.005):
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            s = self.nvml.sample()  # and one as the region ends
            self.stop_evt.set()
            self.t.join(timeout=5)
            if s is not None:
                self.samples.append(s)
            sm = [x[0] for x in self.samples]
            reasons = set().union(*(x[1] for x in self.samples))
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.nvml.max_mhz, "reasons": sorted(reasons),
                    "samples": len(sm), "source": "nvml, 5 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms"}


_PAGE = {}


def host_page():
    import synth
    if "p" not in _PAGE:
        _PAGE["p"] = synth.page(H, W_IMG, SEED, synth.STAINS, CH)
    return _PAGE["p"]


def cpu_oracle_sample(rows: int, threads: int, method: int | None = None, cols: int | None = None, runs=None):
    """Time the oracle (sliding-window path by default) on a rows x cols crop of the page over `runs`."""
    import oracle
    cols = cols or W_IMG
    runs = runs or RUNS
    img = host_page()[:rows, :cols].copy()
    t0 = time.perf_counter()
    for W, rule, k, R in runs:
        oracle.binarize(img, W, oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK, k, R,
                        method=oracle.SLIDING if method is None else method, threads=threads)
    dt = time.perf_counter() - t0
    return rows * cols * len(runs) / dt / 1e6, dt


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    rows = 512
    for _ in range(args.warmup):
        cpu_oracle_sample(rows, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_sample(rows, threads)
    dt = time.perf_counter() - t0
    value = args.steps * rows * W_IMG * len(RUNS) / dt / 1e6
    sample = f"{rows}x4096 RGB crop of the page per step, all 8 (rule, W) runs, oracle sliding path"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (CPU oracle on a crop)"},
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1210_3165_gb300 as bnz

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    bnz.load()
    dev = torch.device("cuda", local)
    page = host_page()
    srcs = []
    for _ in range(NCOPY):
        srcs.append(bnz.to_device_pitched(page, dev))
    outs = [bnz.alloc_pitched(H, W_IMG, dev) for _ in range(NCOPY)]
    stream = torch.cuda.Stream(device=dev)
    rule_id = {"sauvola": bnz.BNZ_SAUVOLA, "niblack": bnz.BNZ_NIBLACK}

    rot = [0]

    def launch(j):
        W, rule, k, R = RUNS[j]
        c = rot[0] % NCOPY
        rot[0] += 1
        bnz.bnz_binarize_dev(srcs[c], W, rule_id[rule], k, R, outs[c], stream=stream)

    def step():
        # every launch reads the next of the NCOPY input copies, so none finds its input in L2
        for j in range(len(RUNS)):
            launch(j)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    # timed region: passes of exactly K steps, each bracketed by an event pair and a
    # synchronize, repeated until at least --min-seconds have passed (so the clock record
    # has samples under load); the job's time per pass is the median pass
    clocks = ClockSampler(local, gpu_uuid(dev))
    clocks.start()
    pass_ms = []
    t_start = time.perf_counter()
    while True:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            for _ in range(args.steps):
                step()
            b.record(stream)
        stream.synchronize()
        pass_ms.append(a.elapsed_time(b))
        if time.perf_counter() - t_start >= args.min_seconds or len(pass_ms) >= 2000:
            break
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = statistics.median(pass_ms)
    total_ms = max_over_ranks(total_ms, world, dev)

    # per-W times: blocks of BLOCK back-to-back launches of one run between one event pair
    # (lifts the per-launch figure above the event timer's resolution), median of 5 blocks
    BLOCK = 20
    per_block = {j: [] for j in range(len(RUNS))}
    with torch.cuda.stream(stream):
        for _ in range(5):
            for j in range(len(RUNS)):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(BLOCK):
                    launch(j)
                b.record(stream)
                per_block[j].append((a, b))
    stream.synchronize()

    px_step = H * W_IMG * len(RUNS)
    value = job_value(world, args.steps, px_step, total_ms)
    peak, peak_kind = measured_peak()
    bytes_launch = H * W_IMG * BYTES_PER_PX
    per_w = {}
    launch_ms = []
    for j, (W, rule, k, R) in enumerate(RUNS):
        ms = statistics.median(a.elapsed_time(b) / BLOCK for a, b in per_block[j])
        launch_ms.append(ms)
        gbs = bytes_launch / (ms / 1e3) / 1e9
        per_w[f"{rule}_W{W}"] = {"us": round(ms * 1e3, 2), "Mpixel/s": round(H * W_IMG / (ms / 1e3) / 1e6, 1),
                                 "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
    avg_launch_ms = total_ms / (args.steps * len(RUNS))
    achieved = bytes_launch / (avg_launch_ms / 1e3) / 1e9

    result = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "h": H, "w": W_IMG, "channels": CH, "runs_per_step": len(RUNS),
                   "l2": "each launch reads its own input copy (8 copies, 400 MB > 129 MB L2)",
                   "parallelism": f"replicas x{world}"},
        "timing": {"passes": len(pass_ms), "steps_per_pass": args.steps,
                   "ms_per_pass": {"median": total_ms, "min": min(pass_ms), "max": max(pass_ms)},
                   "timed_seconds": round(sum(pass_ms) / 1e3, 3),
                   "per_W": f"blocks of {BLOCK} back-to-back launches per run, median of 5 blocks"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": ncu_traffic(),
                     "kernel": "fused_kernel", "algorithmic_bytes_per_launch": bytes_launch,
                     "peak_kind": peak_kind},
        "per_W": per_w,
        "gpu_launches": len(pass_ms) * args.steps * len(RUNS),
        "clocks": clk,
    }

    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e_host_api(bnz, page, 7)
    if not args.case:
        result["dual"] = dual_runs(bnz, srcs, outs, stream, dev, args.steps, max(args.warmup, 3))
        result["otsu"] = otsu_runs(bnz, srcs, outs, stream, dev, args.steps, max(args.warmup, 3))
        result["gs"] = gs_runs(bnz, srcs, outs, stream, dev)
    if not args.case and not args.no_extra and rank == 0:
        del srcs, outs
        torch.cuda.empty_cache()
        result["config1"] = config1_latency(bnz, dev)
        result["config3"] = config3_large(bnz, dev)
        result["out_of_core"] = out_of_core(bnz)
        result["batch"] = batch_summary(bnz, dev)
        result["serve"] = serve_summary(bnz, args)
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        threads = os.cpu_count() or 1
        v, dt = cpu_oracle_sample(H, threads)
        v1, dt1 = cpu_oracle_sample(256, 1)
        vn, dtn = cpu_oracle_sample(512, threads, method=oracle.NAIVE, cols=512, runs=[RUNS[0], RUNS[3]])
        result["cpu_baseline"] = {"value": v, "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                                  "sample": f"the whole page, all 8 runs, sliding-window path, {dt:.1f} s wall",
                                  "single_thread": {"value": v1, "sample": f"256-row crop, all 8 runs, {dt1:.1f} s"},
                                  "naive_all_cores": {"value": vn, "sample": f"512x512 crop, Sauvola W=15 and W=101, "
                                                                             f"O(W^2) per pixel, {dtn:.1f} s"}}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))
    return 0


def dual_runs(bnz, srcs, outs, stream, dev, steps, warmup):
    """Both rules per W from one kernel (bnz_dual_dev): one launch per W writes the Sauvola (k=0.5, R=128) and the
    Niblack (k=-0.2) mask; each W timed as blocks of 20 back-to-back launches (own input copy each), median of 5."""
    import torch
    Ws = sorted({W for W, _, _, _ in RUNS})
    outs2 = [bnz.alloc_pitched(H, W_IMG, dev) for _ in range(NCOPY)]
    rot = [0]

    def launch(W):
        c = rot[0] % NCOPY
        rot[0] += 1
        bnz.bnz_dual_dev(srcs[c], W, 0.5, 128.0, -0.2, outs[c], outs2[c], stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            for W in Ws:
                launch(W)
    stream.synchronize()
    per = {}
    with torch.cuda.stream(stream):
        ev = {W: [] for W in Ws}
        for _ in range(5):
            for W in Ws:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(20):
                    launch(W)
                b.record(stream)
                ev[W].append((a, b))
    stream.synchronize()
    peak, _ = measured_peak()
    bytes_launch = H * W_IMG * (CH + 2)
    total = 0.0
    for W in Ws:
        ms = statistics.median(a.elapsed_time(b) / 20 for a, b in ev[W])
        total += ms
        per[f"W{W}"] = {"us": round(ms * 1e3, 2), "frac": round(bytes_launch / (ms / 1e3) / 1e9 / peak, 4)}
    masks = len(Ws) * 2 * H * W_IMG
    return {"kernel": "dual_kernel", "launches_per_step": len(Ws), "masks_per_step": 2 * len(Ws),
            "ms_per_step": total, "Mpixel/s": masks / (total / 1e3) / 1e6, "per_W": per,
            "algorithmic_bytes_per_launch": bytes_launch,
            "note": "the same 8 masks as a step of the single-rule runs, two per launch from one pass over the "
                    "window sums; every mask equals the single-rule kernel's"}


def _block_ms(fn, stream, n, reps=5):
    """Median over `reps` blocks of n back-to-back calls between one event pair, in ms per call."""
    import torch
    out = []
    with torch.cuda.stream(stream):
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                fn()
            b.record(stream)
            out.append((a, b))
    stream.synchronize()
    return statistics.median(a.elapsed_time(b) / n for a, b in out)


def config1_latency(bnz, dev):
    """512x512 gray page, Sauvola W=15 k=0.5 R=128: device latency of one launch (events around each launch,
    median of 200), back-to-back throughput, and the host-pointer call's latency (copies included)."""
    import numpy as np
    import torch
    import synth
    img = synth.page(512, 512, 1)
    src = bnz.to_device_pitched(img, dev)
    out = bnz.alloc_pitched(512, 512, dev)
    stream = torch.cuda.Stream(device=dev)

    def call():
        bnz.bnz_binarize_dev(src, 15, bnz.BNZ_SAUVOLA, 0.5, 128.0, out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(20):
            call()
    stream.synchronize()
    lat = []
    for _ in range(200):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            call()
            b.record(stream)
        stream.synchronize()
        lat.append(a.elapsed_time(b))
    tput_ms = _block_ms(call, stream, 200, 3)
    host = np.ascontiguousarray(img)
    hdst = np.empty((512, 512), np.uint8)
    lib = bnz.load()
    hl = []
    for i in range(220):
        t0 = time.perf_counter()
        rc = lib.bnz_sauvola(host.ctypes.data, 512, 512, 1, 15, 0.5, 128.0, hdst.ctypes.data)
        hl.append(time.perf_counter() - t0)
        if rc != 0:
            raise RuntimeError(bnz.bnz_last_error())
    hl = hl[20:]
    return {"workload": "512x512 gray page (seed 1), Sauvola W=15 k=0.5 R=128, byte mask",
            "device_latency_us": {"median": round(statistics.median(lat) * 1e3, 2), "p99": round(sorted(lat)[197] * 1e3, 2),
                                  "calls": 200},
            "back_to_back_us_per_launch": round(tput_ms * 1e3, 2),
            "Mpixel/s_back_to_back": round(512 * 512 / (tput_ms / 1e3) / 1e6, 1),
            "host_call_latency_us": {"median": round(statistics.median(hl) * 1e6, 1), "calls": 200,
                                     "api": "bnz_sauvola, pageable host buffers, copies included"}}


def integral_traffic():
    """DRAM bytes per launch of the integral-image path from the committed ncu summary (same source only)."""
    p = os.path.join(ROOT, "profiles", "integral_traffic.json")
    try:
        d = json.load(open(p))
        h = hashlib.sha256()
        for f in ("integral.cu", "decide.cuh"):
            h.update(open(os.path.join(ROOT, "paper_1210_3165_gb300", "csrc", f), "rb").read())
        if d.get("source_sha") == h.hexdigest()[:16]:
            return d
    except Exception:
        pass
    return None


def config3_large(bnz, dev):
    """16384x16384 gray page (vignetting, sigma 15), Sauvola W=101 k=0.34 R=128: the fused kernel (int32 sums)
    and the integral-image comparison path (int64 tables), each as blocks of back-to-back launches."""
    import torch
    import synth
    h = w = 16384
    img = synth.page(h, w, 3, synth.VIGNETTE, 1)
    src = bnz.to_device_pitched(img, dev)
    del img
    out = bnz.alloc_pitched(h, w, dev)
    stream = torch.cuda.Stream(device=dev)
    peak, _ = measured_peak()

    def fused():
        bnz.bnz_binarize_dev(src, 101, bnz.BNZ_SAUVOLA, 0.34, 128.0, out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(3):
            fused()
    ms_f = _block_ms(fused, stream, 10, 3)
    nbytes = h * w * 2
    res = {"workload": "16384x16384 gray page (seed 3, vignetting, sigma 15), Sauvola W=101 k=0.34 R=128, byte mask",
           "fused": {"ms": round(ms_f, 4), "Mpixel/s": round(h * w / (ms_f / 1e3) / 1e6, 1),
                     "GB/s": round(nbytes / (ms_f / 1e3) / 1e9, 1),
                     "frac": round(nbytes / (ms_f / 1e3) / 1e9 / peak, 4), "algorithmic_bytes": nbytes,
                     "sums": "int32 window sums"}}
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(h, w), dev)

    def integral():
        bnz.bnz_binarize_integral_dev(src, 101, bnz.BNZ_SAUVOLA, 0.34, 128.0, out, scratch, stream=stream)
    with torch.cuda.stream(stream):
        integral()
    ms_i = _block_ms(integral, stream, 3, 3)
    tr = integral_traffic()
    res["integral"] = {"ms": round(ms_i, 4), "Mpixel/s": round(h * w / (ms_i / 1e3) / 1e6, 1),
                       "scratch_bytes": int(scratch.numel()), "sums": "int64 integral images",
                       "dram_bytes_per_call": (tr or {}).get("dram_bytes_per_call"),
                       "dram_bytes_source": (tr or {}).get("source"),
                       "fused_speedup": round(ms_i / ms_f, 2)}
    del scratch, src, out
    torch.cuda.empty_cache()
    return res


def out_of_core(bnz):
    """The 16384x16384 gray page (Sauvola W=101 k=0.34 R=128) from pinned host memory to a pinned host mask:
    the host call (bnz_sauvola, which streams a page of 256 MiB or more through band slots of a quarter of its
    bytes) against the out-of-core call (bnz_binarize_window) through device windows of 1/4 and 1/16 of the
    page + mask bytes.  Copies inside the timed region (the host link bounds all: 268 MB up, 268 MB down)."""
    import torch
    import synth
    h = w = 16384
    src = torch.empty((h, w), dtype=torch.uint8, pin_memory=True)
    synth.page(h, w, 3, synth.VIGNETTE, 1, out=src.numpy())
    dst = torch.empty((h, w), dtype=torch.uint8, pin_memory=True)
    lib = bnz.load()
    sp, dp = src.numpy(), dst.numpy()

    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    def check(rc):
        if rc != 0:
            raise RuntimeError(bnz.bnz_last_error())
    res = {"workload": "16384x16384 gray page, Sauvola W=101 k=0.34 R=128, pinned host page in, pinned host mask out",
           "h2d_bytes_per_call": h * w, "d2h_bytes_per_call": h * w}
    t = timed(lambda: check(lib.bnz_sauvola(sp.ctypes.data, h, w, 1, 101, 0.34, 128.0, dp.ctypes.data)))
    res["host_call"] = {"ms": round(t * 1e3, 2), "Mpixel/s": round(h * w / t / 1e6, 1), "api": "bnz_sauvola"}
    ref = dp.copy()
    for frac in (4, 16):
        win = 2 * h * w // frac
        t = timed(lambda: check(lib.bnz_binarize_window(sp.ctypes.data, h, w, 1, 101, bnz.BNZ_SAUVOLA, 0.34, 128.0,
                                                        dp.ctypes.data, win)))
        res[f"window_1_{frac}"] = {"ms": round(t * 1e3, 2), "Mpixel/s": round(h * w / t / 1e6, 1), "window_bytes": win,
                                   "same_mask_as_host_call": bool((dp == ref).all())}
    return res


def batch_summary(bnz, dev):
    """Config 4: 256 uneven gray pages in one persistent launch replayed from a CUDA graph, against one plain
    launch per page (same pages, same stream)."""
    import torch
    import synth
    from paper_1210_3165_gb300 import tune
    specs = synth.batch_specs(256, seed=4)
    table = tune.load_table()
    pages, px = [], 0
    for sp in specs:
        img = synth.page(sp["h"], sp["w"], sp["seed"], synth.DOC, 1, random_dir=True)
        pages.append(dict(src=bnz.to_device_pitched(img, dev), dst=bnz.alloc_pitched(sp["h"], sp["w"], dev),
                          W=sp["W"], rule="sauvola", k=0.5, R=128.0, tile_w=tune.tile_for(table, 1, sp["W"])))
        px += sp["h"] * sp["w"]
    batch = bnz.Batch(pages, use_graph=True)
    stream = torch.cuda.Stream(device=dev)

    def run_batch():
        batch.run(stream)

    def per_page():
        for pg in pages:
            bnz.bnz_binarize_dev(pg["src"], pg["W"], bnz.BNZ_SAUVOLA, 0.5, 128.0, pg["dst"], stream=stream)
    with torch.cuda.stream(stream):
        run_batch()
        per_page()
    ms_b = _block_ms(run_batch, stream, 3, 5)
    ms_p = _block_ms(per_page, stream, 1, 3)
    peak, _ = measured_peak()
    gbs = px * 2 / (ms_b / 1e3) / 1e9
    info = batch.info()
    batch.close()
    del pages
    torch.cuda.empty_cache()
    return {"workload": BATCH_WORKLOAD, "pages": len(specs), "pixels": px,
            "batched": {"ms": round(ms_b, 3), "pages_per_s": round(len(specs) / (ms_b / 1e3), 1),
                        "Mpixel/s": round(px / (ms_b / 1e3) / 1e6, 1), "frac": round(gbs / peak, 4),
                        "launches": info.get("launches")},
            "per_page_launches": {"ms": round(ms_p, 3), "pages_per_s": round(len(specs) / (ms_p / 1e3), 1),
                                  "Mpixel/s": round(px / (ms_p / 1e3) / 1e6, 1)},
            "speedup_vs_per_page": round(ms_p / ms_b, 3), "tile_table": "cached" if table else "library default"}


def serve_summary(bnz, args):
    """Config 5 on a reduced request count: the native serving engine, batched steps vs one plain launch per
    page, pages from pinned host memory ("host") and already on the device ("resident"): closed-loop capacity
    (median of three runs, all three listed), then the Poisson trace at 0.8 of the batched arm's capacity with
    p50/p99 latency."""
    import torch
    import synth
    from paper_1210_3165_gb300.serve import NativeServer
    n = args.extra_serve_requests
    ch, cw = SERVE_CANVAS
    canvases = [torch.from_numpy(synth.page(ch, cw, 50 + j, prof, 3, random_dir=True)).pin_memory()
                for j, prof in enumerate((synth.STAINS, synth.DOC))]
    budget = 16 << 30
    arms = {"batched": lambda: NativeServer(budget, args.max_batch, batched=True, compute_streams=1),
            "per_image": lambda: NativeServer(budget, args.max_batch, batched=False, compute_streams=1)}
    out = {}
    dev_canvases = [c.to("cuda") for c in canvases]
    for mode, cvs in (("host", canvases), ("resident", dev_canvases)):
        reqs = serve_requests(n, 5, cvs)
        res = {}
        for name, mk in arms.items():
            caps = sorted(serve_once(mk, reqs, None, warm=reqs[:48])["pages_per_s"] for _ in range(3))
            res[name] = {"capacity_pages_per_s": round(caps[1], 1), "capacity_runs": [round(c, 1) for c in caps]}
        load = 0.8 * res["batched"]["capacity_pages_per_s"]
        for name, mk in arms.items():
            st = serve_once(mk, reqs, load, warm=reqs[:48])
            res[name].update({"offered_pages_per_s": round(load, 1), "pages_per_s": round(st["pages_per_s"], 1),
                              "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3)})
        out[mode] = res
    del dev_canvases
    torch.cuda.empty_cache()
    return {"workload": SERVE_WORKLOAD, "requests": n, "note": f"the first {n} requests of the 10,000-request "
            "trace (full runs: bench.py --workload serve)", "engine": "native", "modes": out}


def otsu_runs(bnz, srcs, outs, stream, dev, steps, warmup):
    """Eq. 2 with Otsu's threshold on the same page (bnz_otsu_dev: histogram with the selection in its last CTA,
    then the mask; 2 kernels per call),
    each call on its own input copy; algorithmic bytes: two reads of the RGB page and the byte mask."""
    import torch
    scratch = torch.zeros(bnz.BNZ_OTSU_SCRATCH_BYTES, dtype=torch.uint8, device=dev)
    rot = [0]

    def call():
        c = rot[0] % NCOPY
        rot[0] += 1
        bnz.bnz_otsu_dev(srcs[c], outs[c], scratch, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            call()
    stream.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for s in range(steps):
            call()
            evs[s + 1].record(stream)
    stream.synchronize()
    ts = sorted(evs[s].elapsed_time(evs[s + 1]) for s in range(steps))
    ms = ts[len(ts) // 2]
    peak, _ = measured_peak()
    bytes_call = H * W_IMG * (2 * CH + 1)
    gbs = bytes_call / (ms / 1e3) / 1e9
    T = int(scratch[2048:2052].view(torch.int32).item())
    return {"kernels": "otsu_hist (its last CTA picks T), otsu_mask", "launches_per_call": 2, "us_per_call": round(ms * 1e3, 2),
            "Mpixel/s": H * W_IMG / (ms / 1e3) / 1e6, "algorithmic_bytes_per_call": bytes_call,
            "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4), "T": T}


def gs_runs(bnz, srcs, outs, stream, dev):
    """Reduced-set rule of Sec. 2 (Eq. 5, Sauvola k=0.5 R'=128) on the same page for the six structures
    proposed by this library (the paper's Fig. 1 is not available, so the structures and their accuracy are not
    the paper's): time per launch (blocks of 20 launches, each on its own input copy), algorithmic bytes 4 B/px,
    and the F-measure of Eq. 6 against the page's ground-truth stroke mask and against the exact Sauvola mask
    of the same W (counts from the confusion kernel)."""
    import torch
    import synth
    _, gt = synth.page(H, W_IMG, SEED, synth.STAINS, CH, ground_truth=True)
    d_gt = bnz.to_device_pitched(gt, dev)
    exact = bnz.alloc_pitched(H, W_IMG, dev)
    peak, _ = measured_peak()
    bytes_launch = H * W_IMG * BYTES_PER_PX
    rot = [0]
    res = {"kernel": "gs_kernel", "rule": "Sauvola k=0.5 R'=128", "algorithmic_bytes_per_launch": bytes_launch,
           "structures": {}, "exact_sauvola_fm_vs_ground_truth": {},
           "note": "structures proposed here (cross, diagonals, star, frame, frame+cross, frame+diagonals); "
                   "the paper's Fig. 1 is unavailable, so its accuracy figures are not comparable"}
    Ws = (15, 31, 61, 101)
    for W in Ws:
        bnz.bnz_binarize_dev(srcs[0], W, bnz.BNZ_SAUVOLA, 0.5, 128.0, exact, stream=stream)
        stream.synchronize()
        res["exact_sauvola_fm_vs_ground_truth"][f"W{W}"] = round(bnz.fmeasure(exact, d_gt, 0, 1)[0], 5)
        for gs, name in bnz.GS_NAMES.items():
            def call(gs=gs, W=W):
                c = rot[0] % NCOPY
                rot[0] += 1
                bnz.bnz_gs_binarize_dev(srcs[c], W, gs, bnz.BNZ_SAUVOLA, 0.5, 128.0, outs[c], stream=stream)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    call()
            ms = _block_ms(call, stream, 20)
            bnz.bnz_gs_binarize_dev(srcs[0], W, gs, bnz.BNZ_SAUVOLA, 0.5, 128.0, outs[0], stream=stream)
            stream.synchronize()
            gbs = bytes_launch / (ms / 1e3) / 1e9
            res["structures"].setdefault(name, {})[f"W{W}"] = {
                "us": round(ms * 1e3, 2), "Mpixel/s": round(H * W_IMG / (ms / 1e3) / 1e6, 1),
                "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
                "fm_vs_ground_truth": round(bnz.fmeasure(outs[0], d_gt, 0, 1)[0], 5),
                "fm_vs_exact_sauvola": round(bnz.fmeasure(outs[0], exact, 0, 0)[0], 5)}
    return res


def e2e_host_api(bnz, page, steps):
    """Same metric through the host-pointer C ABI, copies inside the timed region: a step uploads the pinned
    page once and brings back its 8 masks with bnz_binarize_runs (one page, eight settings; uploads, kernels and
    downloads overlapped band by band).  Also reported: the same step as 8 one-setting calls (bnz_sauvola /
    bnz_niblack), each uploading the page again."""
    import numpy as np
    import torch
    src = torch.empty(page.shape, dtype=torch.uint8, pin_memory=True)
    src.numpy()[...] = page
    dsts = [torch.empty((H, W_IMG), dtype=torch.uint8, pin_memory=True) for _ in RUNS]
    lib = bnz.load()
    sp = src.numpy()
    arr = (bnz.bnz_run * len(RUNS))()
    for j, (W, rule, k, R) in enumerate(RUNS):
        arr[j] = bnz.bnz_run(W, bnz.BNZ_SAUVOLA if rule == "sauvola" else bnz.BNZ_NIBLACK, k, R,
                             dsts[j].numpy().ctypes.data)

    def runs():
        rc = lib.bnz_binarize_runs(sp.ctypes.data, H, W_IMG, CH, arr, len(RUNS))
        if rc != 0:
            raise RuntimeError(bnz.bnz_last_error())

    def per_call():
        dp = dsts[0].numpy()
        for W, rule, k, R in RUNS:
            if rule == "sauvola":
                rc = lib.bnz_sauvola(sp.ctypes.data, H, W_IMG, CH, W, k, R, dp.ctypes.data)
            else:
                rc = lib.bnz_niblack(sp.ctypes.data, H, W_IMG, CH, W, k, dp.ctypes.data)
            if rc != 0:
                raise RuntimeError(bnz.bnz_last_error())

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts), ts  # the median step is robust to host hiccups

    dt, ts = timed(runs)
    dt1, _ = timed(per_call)
    return {"value": H * W_IMG * len(RUNS) / dt / 1e6, "unit": "Mpixel/s",
            "h2d_bytes_per_step": H * W_IMG * CH, "d2h_bytes_per_step": H * W_IMG * len(RUNS),
            "api": "bnz_binarize_runs (host pointers, pinned): the page up once, its 8 masks down", "steps": steps,
            "ms_per_step": {"median": dt * 1e3, "min": min(ts) * 1e3, "max": max(ts) * 1e3},
            "one_setting_calls": {"value": H * W_IMG * len(RUNS) / dt1 / 1e6, "unit": "Mpixel/s",
                                  "h2d_bytes_per_step": H * W_IMG * CH * len(RUNS),
                                  "d2h_bytes_per_step": H * W_IMG * len(RUNS),
                                  "api": "8 calls of bnz_sauvola / bnz_niblack, each uploading the page"}}


BATCH_WORKLOAD = "batch of 256 uint8 gray pages, width U[600,2480] x height U[800,3508], W from {15,25,45,75}, " \
                 "Sauvola k=0.5 R=128, one persistent launch per run replayed from a CUDA graph, strip widths " \
                 "from the autotuner"


def run_batch(args):
    """Uneven-page batch: graph-replayed persistent launch vs one plain launch per page."""
    import torch
    import synth
    import paper_1210_3165_gb300 as bnz
    from paper_1210_3165_gb300 import tune
    torch.cuda.set_device(0)
    bnz.load()
    specs = synth.batch_specs(256, seed=4)
    table = tune.load_table() or tune.tune(windows=(15, 25, 45, 75), channels=(1,), reps=5)
    pages, px = [], 0
    for sp in specs:
        img = synth.page(sp["h"], sp["w"], sp["seed"], synth.DOC, 1, random_dir=True)
        pages.append(dict(src=bnz.to_device_pitched(img), dst=bnz.alloc_pitched(sp["h"], sp["w"]), W=sp["W"],
                          rule="sauvola", k=0.5, R=128.0, tile_w=tune.tile_for(table, 1, sp["W"])))
        px += sp["h"] * sp["w"]
    batch = bnz.Batch(pages, use_graph=True)
    stream = torch.cuda.Stream()

    def timed(fn, steps, warmup, clocks=None):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks is not None:
            clocks.start()
        with torch.cuda.stream(stream):
            a.record(stream)
            for _ in range(steps):
                fn()
            b.record(stream)
        stream.synchronize()
        if clocks is not None:
            clocks.result = clocks.stop()
        return a.elapsed_time(b) / steps

    clocks = ClockSampler(torch.cuda.current_device(), gpu_uuid(torch.cuda.current_device()))
    ms_batch = timed(lambda: batch.run(stream), args.steps, max(args.warmup, 3), clocks)

    def per_page():
        for pg in pages:
            bnz.bnz_binarize_dev(pg["src"], pg["W"], bnz.BNZ_SAUVOLA, 0.5, 128.0, pg["dst"], stream=stream)
    ms_pages = timed(per_page, max(1, args.steps // 4), 2)
    peak, peak_kind = measured_peak()
    gbs = px * 2 / (ms_batch / 1e3) / 1e9
    print(json.dumps({
        "metric": METRIC, "value": px / (ms_batch / 1e3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "pages": len(pages), "pixels": px, "launches_per_run": 1,
                   "l2": "working set 1.7 GB > 129 MB L2"},
        "pages_per_s": len(pages) / (ms_batch / 1e3),
        "per_page_launches": {"ms_per_batch": ms_pages, "pages_per_s": len(pages) / (ms_pages / 1e3),
                              "Mpixel/s": px / (ms_pages / 1e3) / 1e6},
        "speedup_vs_per_page": ms_pages / ms_batch,
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "traffic": None, "peak_kind": peak_kind},
        "tiles": table.get("1"), "batch_info": batch.info(), "gpu_launches": args.steps,
        "clocks": getattr(clocks, "result", None),
    }))
    batch.close()
    return 0


SERVE_WORKLOAD = "Poisson stream of uint8 RGB pages, width U[600,4960] x height U[800,7016], W odd U{15..101}, " \
                 "Sauvola k=0.5 R=128 / Niblack k=-0.2 50/50, 16 GB device budget, pages from pinned host memory, " \
                 "byte masks back to pinned host memory"
SERVE_CANVAS = (7016, 4960)


def serve_requests(n, seed, canvases):
    """The trace's requests as crops of pinned host canvases (row pitch = the canvas's)."""
    import numpy as np
    import synth
    trace = synth.serve_trace(n, seed=seed, rate_per_s=1.0)
    rng = np.random.default_rng(seed + 1)
    out = []
    for i, tr in enumerate(trace):
        cv = canvases[i % len(canvases)]
        y0 = int(rng.integers(0, SERVE_CANVAS[0] - tr["h"] + 1))
        x0 = int(rng.integers(0, SERVE_CANVAS[1] - tr["w"] + 1)) // 16 * 16   # 16-byte aligned device crops
        out.append((tr, cv[y0:y0 + tr["h"], x0:x0 + tr["w"]]))
    return out


def serve_once(make_server, reqs, rate, warm=()):
    """Replay `reqs` through a fresh server (rate None: all at once, closed loop); pages/s and latency stats.
    `warm` requests go through the same server first (closed loop, waited for, not counted): the measured trace
    then meets a running server, as in service, not one in its first milliseconds."""
    from paper_1210_3165_gb300.serve import Request
    srv = make_server()
    base = {}
    if warm:
        futs = []
        for tr, img in warm:
            r = Request(image=img, W=tr["W"], rule=tr["rule"], k=tr["k"], R=tr["R"])
            srv.submit(r)
            futs.append(r.future)
        for f in futs:
            f.result()
        futs = r = None  # their masks go back to the server's host arena
        while srv.pending():
            time.sleep(1e-3)
        base = srv.stats()
        srv.latencies.clear()  # every warm request has completed: the poller adds no more of theirs
    done_t = []
    t0 = time.perf_counter() + 0.01
    for tr, img in reqs:
        due = t0 + (tr["t"] / rate if rate else 0.0)
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        r = Request(image=img, W=tr["W"], rule=tr["rule"], k=tr["k"], R=tr["R"], arrival=due)
        r.future.add_done_callback(lambda f: done_t.append(time.perf_counter()))
        srv.submit(r)
    srv.stop(drain=True)
    st = srv.stats()
    for key in ("completed", "steps", "alloc_waits"):
        if key in base:
            st[key] -= base[key]
    span = max(done_t) - t0
    st.update(pages_per_s=len(reqs) / span, seconds=span, offered_pages_per_s=rate,
              mpix_per_s=sum(tr["h"] * tr["w"] for tr, _ in reqs) / span / 1e6, warm_requests=len(warm))
    return st


def run_serve(args):
    """Continuous-batching server vs per-image launches on a Poisson stream of RGB pages, for the native
    engine (C++ scheduler) and the Python loop."""
    import torch
    import synth
    import paper_1210_3165_gb300 as bnz
    from paper_1210_3165_gb300.serve import NativeServer, Server, TorchExecutor
    torch.cuda.set_device(0)
    bnz.load()
    ch, cw = SERVE_CANVAS
    canvases = []
    for j, prof in enumerate((synth.STAINS, synth.DOC, synth.VIGNETTE, synth.STAINS)):
        canvases.append(torch.from_numpy(synth.page(ch, cw, 50 + j, prof, 3, random_dir=True)).pin_memory())
    n = args.serve_requests
    budget = 16 << 30
    loads = [float(x) for x in args.serve_loads.split(",")]
    engines = ["native", "python"] if args.serve_engine == "both" else [args.serve_engine]
    makers = {}
    if "native" in engines:
        makers["native"] = {
            "batched": lambda: NativeServer(budget, args.max_batch, batched=True, compute_streams=1),
            "per_image": lambda: NativeServer(budget, args.max_batch, batched=False, compute_streams=1)}
    if "python" in engines:
        exs = {"batched": TorchExecutor(batched=True, compute_streams=1, budget_bytes=budget),
               "per_image": TorchExecutor(batched=False, budget_bytes=budget)}
        makers["python"] = {name: (lambda ex=ex: Server(ex, max_batch=args.max_batch).start())
                            for name, ex in exs.items()}
    results = {}
    # "host": pages in pinned host memory, H2D + kernel + D2H per request;
    # "resident": pages already in device memory (crops of device canvases), kernel + D2H
    dev_canvases = [c.to("cuda") for c in canvases]
    for engine, arms in makers.items():
        modes = {}
        for mode, cvs in (("host", canvases), ("resident", dev_canvases)):
            reqs = serve_requests(n, 5, cvs)
            res = {}
            for name, mk in arms.items():
                res[name] = {"capacity": serve_once(mk, reqs[:min(n, args.serve_capacity)], None, warm=reqs[:64]),
                             "loads": []}
            cap_b = res["batched"]["capacity"]["pages_per_s"]
            for name, mk in arms.items():
                for ld in loads:
                    st = serve_once(mk, reqs, ld * cap_b, warm=reqs[:64])
                    st["load"] = ld
                    res[name]["loads"].append(st)
            modes[mode] = res
        results[engine] = modes
    head = results[engines[0]]["host"]
    top = head["batched"]["loads"][-1]
    px = sum(tr["h"] * tr["w"] for tr, _ in reqs)
    print(json.dumps({
        "metric": METRIC, "value": round(top["pages_per_s"], 2), "unit": "pages/s", "n_gpus": 1,
        "steps": n, "warmup": 64, "ms_per_step": 1e3 / top["pages_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "requests": n, "mean_mpix_per_page": round(px / n / 1e6, 3),
                   "budget_bytes": budget, "max_batch": args.max_batch, "loads_of_batched_capacity": loads,
                   "engine": engines[0], "l2": "pages of 1.4-104 MB stream through; working set >> 129 MB L2"},
        "p50_ms": round(top["p50_ms"], 3), "p99_ms": round(top["p99_ms"], 3),
        "e2e": {"value": round(top["pages_per_s"], 2), "unit": "pages/s",
                "h2d_bytes_per_step": px * 3 // n, "d2h_bytes_per_step": px // n},
        "serve": results, "gpu_launches": top["steps"],
        "device_memory_reserved_max": torch.cuda.max_memory_reserved(),
    }))
    return 0


def run_integral(args):
    """The integral-image comparison path alone on an N x N gray page (vignetting, sigma 15), Sauvola W=101
    k=0.34 R=128: --warmup calls, then --steps timed calls (for profiler captures of one call)."""
    import torch
    import synth
    import paper_1210_3165_gb300 as bnz
    torch.cuda.set_device(0)
    bnz.load()
    n = args.integral_size
    img = synth.page(n, n, 3, synth.VIGNETTE, 1)
    src = bnz.to_device_pitched(img)
    out = bnz.alloc_pitched(n, n)
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(n, n))
    stream = torch.cuda.Stream()

    def call():
        bnz.bnz_binarize_integral_dev(src, 101, bnz.BNZ_SAUVOLA, 0.34, 128.0, out, scratch, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            call()
    ms = _block_ms(call, stream, max(args.steps, 1), 1)
    print(json.dumps({"workload": f"integral-image path, {n}x{n} gray page, Sauvola W=101 k=0.34 R=128",
                      "ms_per_call": ms, "Mpixel/s": n * n / (ms / 1e3) / 1e6, "kernels_per_call": 5}))
    return 0


def run_gs(args):
    """The reduced-set kernel alone (Sec. 2, Eq. 5, Sauvola k=0.5 R'=128) on the 4096x4096 RGB page for one
    structure and W (--gs-case GS,W): --warmup calls, then --steps timed calls (for profiler captures)."""
    import torch
    import paper_1210_3165_gb300 as bnz
    torch.cuda.set_device(0)
    bnz.load()
    gs, W = (int(v) for v in args.gs_case.split(","))
    src = bnz.to_device_pitched(host_page())
    out = bnz.alloc_pitched(H, W_IMG)
    stream = torch.cuda.Stream()

    def call():
        bnz.bnz_gs_binarize_dev(src, W, gs, bnz.BNZ_SAUVOLA, 0.5, 128.0, out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            call()
    ms = _block_ms(call, stream, max(args.steps, 1), 1)
    print(json.dumps({"workload": f"reduced set {bnz.GS_NAMES[gs]}, W={W}, {WORKLOAD.split(',')[0]}",
                      "ms_per_call": ms, "Mpixel/s": H * W_IMG / (ms / 1e3) / 1e6, "kernels_per_call": 1}))
    return 0


def run_edge_sweep(args):
    """Fused kernel time per launch against bnz_tile.edge_weight on the page workload (blocks of 20 launches,
    median of 7, each launch on its own input copy): the sweep behind the library's default edge weight."""
    import torch
    import paper_1210_3165_gb300 as bnz
    torch.cuda.set_device(0)
    bnz.load()
    page = host_page()
    srcs = [bnz.to_device_pitched(page) for _ in range(NCOPY)]
    outs = [bnz.alloc_pitched(H, W_IMG) for _ in range(NCOPY)]
    stream = torch.cuda.Stream()
    rot = [0]
    res = {}
    for W, rule, k, R in RUNS:
        row = {}
        rid = bnz.BNZ_SAUVOLA if rule == "sauvola" else bnz.BNZ_NIBLACK
        for ew in (16, 18, 20, 22, 24, 28, 32):
            tile = bnz.bnz_tile(0, 0, 0, ew)

            def call():
                c = rot[0] % NCOPY
                rot[0] += 1
                bnz.bnz_binarize_dev(srcs[c], W, rid, k, R, outs[c], tile=tile, stream=stream)
            with torch.cuda.stream(stream):
                for _ in range(max(args.warmup, 3)):
                    call()
            row[ew] = round(_block_ms(call, stream, 20, 7) * 1e3, 2)
        res[f"{rule}_W{W}"] = row
    print(json.dumps({"workload": WORKLOAD, "us_per_launch_by_edge_weight": res}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other configurations' keys")
    ap.add_argument("--min-seconds", type=float, default=1.0,
                    help="repeat the K-step timed pass until this much time has passed (median pass reported)")
    ap.add_argument("--workload", default="page", choices=["page", "batch", "serve", "integral", "gs", "edge-sweep"],
                    help="page: the 4096x4096 RGB page (default); batch: 256 uneven gray pages; "
                         "serve: Poisson stream of RGB pages through the serving loop")
    ap.add_argument("--case", default=None,
                    help="page workload restricted to one configuration CH,W,RULE (e.g. 3,15,sauvola): "
                         "one launch per step, for profiler captures")
    ap.add_argument("--integral-size", type=int, default=8192, help="page side of --workload integral")
    ap.add_argument("--gs-case", default="1,31", help="structure and W of --workload gs (e.g. 5,101)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-capacity", type=int, default=2000, help="requests of the closed-loop capacity run")
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95", help="offered loads, fractions of batched capacity")
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--extra-serve-requests", type=int, default=1000,
                    help="requests of the serving summary in the default page run")
    ap.add_argument("--serve-engine", default="both", choices=["native", "python", "both"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "gs":
        return run_gs(args)
    if args.workload == "edge-sweep":
        return run_edge_sweep(args)
    if args.workload == "integral":
        return run_integral(args)
    if args.case:
        global CH, RUNS, NCOPY, BYTES_PER_PX, WORKLOAD
        ch, W, rule = args.case.split(",")
        CH = int(ch)
        k = 0.5 if rule == "sauvola" else -0.2
        RUNS = [(int(W), rule, k, 128.0)]
        NCOPY = 8
        BYTES_PER_PX = CH + 1
        WORKLOAD = f"page 4096x4096 {'RGB' if CH == 3 else 'gray'}, {rule} k={k} W={W}, byte mask (one case)"
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

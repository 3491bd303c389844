#!/usr/bin/env python3
"""Benchmark: 128-bit NTT butterflies/s (and BLAS modmul/s) on one GB300, batched vs plain.

Default workload (one "step"): 256 independent negacyclic NTTs of N = 2^16 under a seeded 124-bit
prime q = 1 mod 2^17, forward then inverse, in place in HBM, through the C ABI.  The timed `value`
is the batched persistent form (mqntt_batch.h: 256 forward jobs and 256 inverse jobs, each inverse
waiting for its forward, one persistent kernel replayed from a CUDA graph); beside it are the
same work as one ntt_forward + one ntt_inverse call over the whole batch ("batched_call") and as
one call per polynomial ("plain").  BLAS (vadd, vsub, vmul, axpy at n = 2^24, 60- and 124-bit) is reported as an
extra block.  One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mq|reference] [--bits 124|60]
                  [--order bitrev|natural] [--no-blas] [--no-cpu-baseline]

--impl reference times the CPU oracle (oracle/, the plain reference of this library) on the same
workload: each step is a bounded sample of the 256 transforms run on the host's cores.
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

METRIC = "128-bit NTT butterflies/s & BLAS modmul/s, batched vs plain on 1 GB300, bit-exact"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
# steps of the pipelined end-to-end job: its fill (the first input copy) and drain (the last result
# copy) are paid once per job, as in a serving loop that runs continuously
E2E_STEPS = 32
E2E_JOBS = 3      # the e2e figure is the median of this many jobs (the host link's rate varies)
# algorithmic 32-bit multiply instructions (lo and hi halves of 32 x 32 limb products) per Shoup
# product: 124-bit residues 30 limb products = 60; 64-bit residues: lo(a w) 4 + hi(a w') 8 + lo(qhat q) 4
MADS_PER_SHOUP = {1: 16, 2: 60}
MADS_PER_BARRETT = {1: 20, 2: 72}


_T0 = time.time()


def progress(msg: str):
    """One line on stderr per phase of the run (the JSON line alone goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def brv(i: int, bits: int) -> int:
    return int(format(i, f"0{bits}b")[::-1], 2) if bits else 0


def residue_int(row, width: int) -> int:
    """Python int of one residue (a uint64 scalar or a row of `width` words, low first)."""
    if width == 1:
        return int(row)
    return sum(int(row[k]) << (64 * k) for k in range(width))


def check_forward_samples(M, torch, dev, sh, plan, x_host, wl, bitrev, opts, n_poly=8, per_poly=8):
    """The forward transform of the timed batched form, checked on its own: the batch's forward jobs
    (the same kernel instantiation and work items as in the timed step) run once on a copy of the
    input; the whole output must equal ntt_forward's, and n_poly x per_poly sampled outputs (plus
    both ends of each sampled polynomial) must equal the oracle's O(N) evaluation of the sum
    definition.  Returns (ok, samples checked, equal to the call form)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    N, batch, width, log2n = wl["N"], wl["batch"], wl["width"], wl["log2n"]
    dv, dc = M.to_device(x_host, dev), M.to_device(x_host, dev)
    jobs = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, plan, dv[b * N:(b + 1) * N], 1, N) for b in range(batch)]
    fb = M.mq_batch_create(jobs, opts, stream=sh)
    M.mq_batch_launch(fb, stream=sh)
    status = M.mq_batch_status(fb)
    M.ntt_forward(plan, dc, batch, N, stream=sh)
    torch.cuda.synchronize()
    got, call = M.to_host(dv), M.to_host(dc)
    same_as_call = bool(np.array_equal(got, call))
    del fb, dv, dc
    shp = (batch, N) if width == 1 else (batch, N, width)
    g, xs = got.reshape(shp), x_host.reshape(shp)
    rng = np.random.default_rng(99)
    polys = sorted(int(p) for p in rng.choice(batch, size=min(n_poly, batch), replace=False))
    tasks = []
    for p in polys:
        for i in sorted({0, N - 1} | {int(v) for v in rng.choice(N, size=per_poly, replace=False)}):
            k = brv(i, log2n) if bitrev else i
            tasks.append((p, i, k))
    O = oracle.default()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        want = list(ex.map(lambda t: O.ntt_point(xs[t[0]], log2n, wl["q"], wl["psi"], width, t[2]), tasks))
    ok = status == 0 and all(residue_int(g[p, i], width) == w for (p, i, _), w in zip(tasks, want))
    return bool(ok), len(tasks), same_as_call


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mq", choices=["mq", "reference"])
    p.add_argument("--bits", type=int, default=124, choices=[124, 60])
    p.add_argument("--order", default="bitrev", choices=["bitrev", "natural"])
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--log2n", type=int, default=16)
    p.add_argument("--no-blas", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--workload", default="uniform", choices=["uniform", "serve", "int8-probe"],
                   help="uniform: the default line (uniform batch, plus BLAS and the uneven batch as extra blocks); "
                        "serve: the Poisson serving sweep")
    p.add_argument("--no-uneven", action="store_true")
    p.add_argument("--no-polymul", action="store_true")
    p.add_argument("--no-wide", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=1.5)
    p.add_argument("--serve-point-seconds", type=float, default=0.5,
                   help="seconds of arrivals per point of the default line's short serving sweep")
    p.add_argument("--no-serve", action="store_true", help="leave the short serving sweep out of the default line")
    p.add_argument("--tune", action="store_true",
                   help="autotune the uniform batch before timing it (its choice on the GB300 equals the library's "
                        "defaults: prefetching form, 3 CTAs per SM, lag 32, even split); the uneven batch is always tuned")
    p.add_argument("--no-other-width", action="store_true",
                   help="leave out the uniform batch at the other residue width (60-bit when --bits 124)")
    p.add_argument("--lag", type=int, default=0, help="pipeline lag of the persistent batch (0: library default)")
    p.add_argument("--ctas-per-sm", type=int, default=0, help="persistent CTAs per SM (0: library default)")
    p.add_argument("--form", choices=["default", "split", "prefetch"], default="default",
                   help="persistent kernel form (default: the library's choice for the batch)")
    p.add_argument("--e2e-buffers", type=int, default=3, help="device buffers of the pipelined end-to-end loop (>= 2)")
    p.add_argument("--int8-n", type=int, nargs="*", default=[4096, 8192, 16384],
                   help="matrix sizes of the int8 / bf16 GEMM probe (--workload int8-probe)")
    return p.parse_args()


# ----------------------------------------------------------------------------------- workload

def workload(args):
    from paper_2509_12494_gb300 import workload as W
    log2n, batch = args.log2n, args.batch
    q = W.gen_prime(args.bits, log2n + 1, 1)
    psi = W.gen_root(q, log2n, 1)
    width = 2 if args.bits > 60 else 1
    return dict(log2n=log2n, N=1 << log2n, batch=batch, q=q, psi=psi, width=width,
                butterflies_per_dir=batch * (1 << (log2n - 1)) * log2n)


def workload_name(wl, args):
    return (f"uniform batched NTT: {wl['batch']} x N=2^{wl['log2n']} negacyclic forward+inverse, "
            f"{args.bits}-bit q = 1 mod 2^{wl['log2n'] + 1}, {args.order} order")


KERNEL_SOURCES = ["residue.cuh", "common.cuh", "ntt_kernel.cuh", "tma.cuh", "blas_ops.cuh", "batch_internal.h",
                  "batch_kernel.cuh", "batch.cu"]


def kernel_sources_sha256() -> str:
    """Hash of the code (comments and blank space removed) of the sources that define the persistent
    kernel, to tell whether a profile is current."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2509_12494_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def profiled_traffic(summary: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current sources."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        fields = {}
        for line in open(path):
            if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_sources_sha256")):
                k, v = line.strip().split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_sources_sha256") == kernel_sources_sha256():
            return float(fields["traffic_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


# ----------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is under load."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        busy = [float(r[1]) for r in self.rows if len(r) > 4 and r[4].isdigit() and int(r[4]) > 0 and
                r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 6 + i and r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(busy or sm) if (busy or sm) else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows),
                "samples_busy": len(busy)}


class NvmlClocks:
    """SM clock and clock-event reasons polled through NVML (read-only queries) every ~0.5 ms from a
    host thread while the timed steps run; the nvidia-smi sampler above is the fallback."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import ctypes
        self.ok, self.rows, self.stop_ev, self.t = False, [], threading.Event(), None
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            import torch
            self.h = ctypes.c_void_p()
            uuid = str(getattr(torch.cuda.get_device_properties(torch_device), "uuid", ""))
            found = False
            if uuid:
                key = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
                found = self.lib.nvmlDeviceGetHandleByUUID(key.encode(), ctypes.byref(self.h)) == 0
            if not found:
                found = self.lib.nvmlDeviceGetHandleByIndex_v2(torch_device.index or 0, ctypes.byref(self.h)) == 0
            self.ok = found
            self.c = ctypes
        except Exception:
            self.ok = False

    def _poll(self):
        c = self.c
        mhz, mx, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
        get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_ev.is_set():
            if (self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(mhz)) == 0 and
                    self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, c.byref(mx)) == 0 and
                    get_reasons(self.h, c.byref(rs)) == 0):
                self.rows.append((mhz.value, mx.value, rs.value))
            time.sleep(0.0005)

    def start(self):
        if self.ok:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()

    def stop(self):
        if self.t:
            self.stop_ev.set()
            self.t.join(timeout=5)

    def summary(self):
        if not self.rows:
            return None
        reasons = sorted({n for _, _, r in self.rows for bit, n in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": reasons, "samples": len(self.rows), "source": "NVML, polled every ~0.5 ms during the timed steps"}


# ----------------------------------------------------------------------------------- replicas

def aggregate(ms_local: float, units_local: float, world: int, device=None):
    """Whole-job throughput of `world` independent replicas (weak scaling): the slowest rank's
    time and all ranks' units; returns (ms, units per second).  No data crosses ranks."""
    if world == 1:
        return ms_local, units_local / (ms_local * 1e-3)
    import torch
    import torch.distributed as dist
    ms = torch.tensor([ms_local], dtype=torch.float64, device=device)
    units = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    ms_max = float(ms.item())
    return ms_max, float(units.item()) / (ms_max * 1e-3)


# ----------------------------------------------------------------------------------- GPU arm

def flush_l2(buf):
    buf.add_(1)  # writes 2 x L2 bytes: evicts the working set between timed steps


def run_gpu(args, rank, world):
    import torch

    from paper_2509_12494_gb300 import mqntt as M
    from paper_2509_12494_gb300 import workload as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    M.load(build_if_missing=True)
    wl = workload(args)
    N, batch, width, q, psi = wl["N"], wl["batch"], wl["width"], wl["q"], wl["psi"]
    flags = M.MQ_ORDER_BITREV if args.order == "bitrev" else M.MQ_ORDER_NATURAL
    stream = torch.cuda.Stream(dev)
    sh = stream.cuda_stream
    plan = M.ntt_plan_create(wl["log2n"], q, psi, width, flags, stream=sh)

    x_host = W.gen_residues(batch * N, q, seed=11 + rank, width=width)
    d = M.to_device(x_host, dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(2 * l2 // 4 + 1024, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def step_call():
        M.ntt_forward(plan, d, batch, N, stream=sh)
        M.ntt_inverse(plan, d, batch, N, stream=sh)

    # the persistent batch: job i = forward of polynomial i, job batch + i = its inverse
    jobs = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, plan, d[b * N:(b + 1) * N], 1, N) for b in range(batch)]
    jobs += [M.ntt_job(M.MQ_JOB_NTT_INVERSE, plan, d[b * N:(b + 1) * N], 1, N, after=b) for b in range(batch)]
    opts = batch_opts(M, args)
    tuned = None
    if opts is None and args.tune:
        # the library's autotuner on this batch shape, through a cache file as a user would run it
        # (it runs the batch, so the input is restored afterwards)
        import tempfile
        progress("autotuning the uniform batch")
        t0 = time.perf_counter()
        with tempfile.TemporaryDirectory() as tdir:
            opts = M.mq_autotune_batch(jobs, os.path.join(tdir, "tune.json"), stream=sh)
        tuned = describe_opts(M, opts)
        tuned["tune_s"] = time.perf_counter() - t0
        d.copy_(M.to_device(x_host, dev))
        torch.cuda.synchronize()
    pbatch = M.mq_batch_create(jobs, opts, stream=sh)
    pinfo = M.mq_batch_info(pbatch)

    def step_batched():
        M.mq_batch_launch(pbatch, stream=sh)

    row = width if width == 2 else 1

    def step_plain():
        for b in range(batch):
            M.ntt_forward(plan, d[b * N:(b + 1) * N], 1, N, stream=sh)
        for b in range(batch):
            M.ntt_inverse(plan, d[b * N:(b + 1) * N], 1, N, stream=sh)

    def timed(step, steps, warmup, sampler=None):
        """Per-step device time (ms) with CUDA events on the launching stream; L2 flushed between."""
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step()
                flush_l2(flush)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            if sampler:
                sampler.start()
            times = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                flush_l2(flush)
                times.append((e0, e1))
            torch.cuda.synchronize()
            if sampler:
                sampler.stop()
            if world > 1:
                torch.distributed.barrier()
        return [a.elapsed_time(b) for a, b in times]

    # per-direction kernel time, for the roofline of the transform kernels
    def timed_dirs(steps):
        fw, iv = [], []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                M.ntt_forward(plan, d, batch, N, stream=sh)
                e[1].record(stream)
                M.ntt_inverse(plan, d, batch, N, stream=sh)
                e[2].record(stream)
                flush_l2(flush)
                fw.append((e[0], e[1]))
                iv.append((e[1], e[2]))
            torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in fw], [a.elapsed_time(b) for a, b in iv]

    progress("timing the batched form")
    nvml = NvmlClocks(dev)
    with ClockSampler(dev.index) as clk:
        t_batched = timed(step_batched, args.steps, args.warmup, nvml)
        clocks = nvml.summary() or clk.summary()
    bfly = 2 * wl["butterflies_per_dir"]
    ms, value = aggregate(sum(t_batched) / len(t_batched), bfly, world, dev)

    # correctness of what was timed: the round trip leaves the input unchanged, and the forward
    # half, run alone by the same kernel, matches the oracle at sampled outputs
    batch_status = M.mq_batch_status(pbatch)
    ok_roundtrip = bool(np.array_equal(M.to_host(d), x_host)) and batch_status == 0
    progress("checking the forward half against the oracle")
    fwd_ok, fwd_n, fwd_call = check_forward_samples(M, torch, dev, sh, plan, x_host, wl, args.order == "bitrev",
                                                    batch_opts(M, args))

    out = {"metric": METRIC, "value": value, "unit": "butterflies/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u128" if width == 2 else "u64", "data": "synthetic",
           "config": {"workload": workload_name(wl, args), "batch": batch, "log2n": wl["log2n"],
                      "q_bits": args.bits, "order": args.order,
                      "form": f"batched persistent kernel in a CUDA graph ({pinfo['items']} work items, "
                              f"{pinfo['ctas']} CTAs)",
                      "batch_options": tuned or "library defaults",
                      "l2": "L2 flushed between timed steps (2 x L2 write); working set "
                            f"{batch * N * 8 * width >> 20} MiB", "parallelism": f"replicas x{world}"},
           "roundtrip_bit_exact": ok_roundtrip, "forward_sampled_bit_exact": fwd_ok,
           "forward_check": {"samples_vs_oracle": fwd_n, "whole_output_equals_call_form": fwd_call,
                             "what": "the batch's forward jobs run alone on a copy of the input; sampled "
                                     "outputs of 8 polynomials vs the oracle's sum definition"}}

    # gpu launches in the timed region: one persistent kernel per step (plus a counter memset and
    # a 4-byte status copy in the same graph)
    passes = 1 if wl["log2n"] <= 12 else 2
    out["gpu_launches"] = args.steps

    if rank != 0:
        return None

    progress("call form and plain calls")
    # the same work as one call per direction over the whole batch
    t_call = timed(step_call, max(3, args.steps), 1)
    ms_call = sum(t_call) / len(t_call)
    out["batched_call"] = {"value": bfly / (ms_call * 1e-3), "unit": "butterflies/s", "ms_per_step": ms_call,
                           "form": f"ntt_forward + ntt_inverse over all {batch} polynomials ({2 * passes} launches)"}

    # plain per-call path
    if not args.no_plain:
        t_plain = timed(step_plain, max(2, args.steps // 2), 1)
        ms_plain = sum(t_plain) / len(t_plain)
        out["plain"] = {"value": bfly / (ms_plain * 1e-3), "unit": "butterflies/s", "ms_per_step": ms_plain,
                        "form": f"{batch} ntt_forward + {batch} ntt_inverse calls of batch 1",
                        "batched_over_plain": ms_plain / ms}

    # roofline of the dominant kernel: the persistent kernel, one launch per step (event-timed
    # median of single-launch steps); the per-pass kernels of the one-call form beside it
    t_roof = timed(step_batched, max(5, args.steps), 1)
    ms_launch = statistics.median(t_roof)
    fw, iv = timed_dirs(max(3, args.steps))
    ms_f, ms_i = statistics.median(fw), statistics.median(iv)
    # algorithmic 32-bit multiply instructions per Shoup product (a lo and a hi half per 32 x 32 limb
    # product): 124-bit q, 30 limb products (10 for the quotient's high half, 10 each for the low
    # halves of a w and qhat q) = 60; 60-bit q, lo(a w) 2 + hi(a w') 8 + lo(qhat q) ... = 16
    mads_per_mul = MADS_PER_SHOUP[width]
    mad_f = wl["butterflies_per_dir"] * mads_per_mul
    mad_i = (wl["butterflies_per_dir"] + batch * N // 2) * mads_per_mul  # + N/2 folded N^-1 products
    alu_achieved = (mad_f + mad_i) / (ms_launch * 1e-3)
    probe = {}
    for kind, name in ((M.MQ_PROBE_MAD_CC, "mad_cc"), (M.MQ_PROBE_MAD_LO, "mad_lo"), (M.MQ_PROBE_MAD_HI, "mad_hi")):
        rate, pms = M.mq_probe_imad_rate(kind, 4000, stream=sh)
        probe[name] = rate
    alu_peak = probe["mad_cc"]
    bytes_per_launch = 2 * passes * 2 * batch * N * 8 * width   # every pass reads and writes each residue
    hbm_peak = measured_peaks().get("hbm_gbs")
    hbm_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or HBM_FALLBACK_GBS
    hbm_achieved = bytes_per_launch / (ms_launch * 1e-3) / 1e9
    alu_frac, hbm_frac = alu_achieved / alu_peak, hbm_achieved / hbm_peak
    kname = "persistent_kernel" if args.form == "split" else "prefetch_kernel"
    traffic = profiled_traffic(f"{kname}_uniform_{batch}x{N}_{args.bits}bit.md")
    kdesc = f"{kname} (the batched form; one launch = one step)"
    if alu_frac >= hbm_frac:
        out["roofline"] = {"bound": "alu", "achieved": alu_achieved / 1e12, "peak": alu_peak / 1e12,
                           "unit": "T mad32/s", "frac": alu_frac,
                           "traffic": traffic, "kernel": kdesc,
                           "peak_source": "measured by mq_probe_imad_rate (carry-chained mad.lo.cc/madc.hi.cc)",
                           "algorithmic": f"{mads_per_mul} 32-bit multiply instructions per Shoup product",
                           "hbm_frac": hbm_frac, "hbm_achieved_gbs": hbm_achieved,
                           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src, "ms_launch": ms_launch}
    else:
        out["roofline"] = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                           "frac": hbm_frac,
                           "traffic": traffic, "kernel": kdesc,
                           "peak_source": hbm_src, "alu_frac": alu_frac, "ms_launch": ms_launch,
                           "alu_achieved_tmads": alu_achieved / 1e12, "alu_peak_tmads": alu_peak / 1e12}
    out["roofline"]["call_form_alu_frac"] = (mad_f + mad_i) / ((ms_f + ms_i) * 1e-3) / alu_peak
    out["roofline"]["call_form_ms_forward"] = ms_f
    out["roofline"]["call_form_ms_inverse"] = ms_i
    out["probe_mad_per_s"] = probe

    # end to end through the public API with host buffers (pinned), copies inside the timed region.
    # Pipelined the way a serving loop would run it: --e2e-buffers device buffers, each with its own
    # batch; a copy stream brings a later step's input in and another takes an earlier step's result
    # out while a step transforms, so every step still copies its 256 MiB in and its result out.  With
    # two buffers step k's input copy waits for step k-2's result copy, which waits for step k-2's
    # transform: the chain transform -> copy out -> copy in -> transform limits the rate, not the
    # link.  A third buffer takes that chain off the critical path.
    nbuf = max(2, args.e2e_buffers)
    host_in = torch.from_numpy(x_host.view(np.int64)).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(nbuf)]
    dbuf = [d] + [torch.empty_like(d) for _ in range(nbuf - 1)]
    pbs = [pbatch]
    for k in range(1, nbuf):
        jk = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, plan, dbuf[k][b * N:(b + 1) * N], 1, N) for b in range(batch)]
        jk += [M.ntt_job(M.MQ_JOB_NTT_INVERSE, plan, dbuf[k][b * N:(b + 1) * N], 1, N, after=b) for b in range(batch)]
        pbs.append(M.mq_batch_create(jk, opts, stream=sh))
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = {(kind, b): torch.cuda.Event() for kind in ("in", "comp", "out") for b in range(nbuf)}

    def e2e_step(k):
        b = k % nbuf
        s_in.wait_event(ev["out", b])              # buffer b's previous result is out
        with torch.cuda.stream(s_in):
            dbuf[b].copy_(host_in.view_as(dbuf[b]), non_blocking=True)
            ev["in", b].record(s_in)
        stream.wait_event(ev["in", b])
        M.mq_batch_launch(pbs[b], stream=sh)
        ev["comp", b].record(stream)
        s_out.wait_event(ev["comp", b])
        with torch.cuda.stream(s_out):
            host_out[b].view_as(dbuf[b]).copy_(dbuf[b], non_blocking=True)
            ev["out", b].record(s_out)

    def e2e_run(steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        s_in.wait_stream(stream)
        for k in range(steps):
            e2e_step(k)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    progress("end to end")
    e2e_run(args.warmup)
    n_e2e = max(E2E_STEPS, args.steps)
    ms_e2e = statistics.median(e2e_run(n_e2e) for _ in range(E2E_JOBS))
    exact = all(np.array_equal(h.numpy().view(np.uint64).reshape(x_host.shape), x_host)
                for h in host_out[:min(nbuf, args.warmup + n_e2e)])

    def step_e2e_serial():
        d.copy_(host_in.view_as(d), non_blocking=True)
        step_batched()
        host_out[0].view_as(d).copy_(d, non_blocking=True)

    def link_run(steps):   # the step's copies alone, both directions at once: the floor of the e2e step
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for k in range(steps):
            with torch.cuda.stream(s_in):
                dbuf[k % nbuf].copy_(host_in.view_as(d), non_blocking=True)
            with torch.cuda.stream(s_out):
                host_out[0].view_as(d).copy_(dbuf[(k + 1) % nbuf], non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    link_run(1)
    ms_link = statistics.median(link_run(n_e2e) for _ in range(E2E_JOBS))

    t_ser = timed(step_e2e_serial, max(3, args.steps // 2), 1)
    ms_ser = sum(t_ser) / len(t_ser)
    torch.cuda.synchronize()
    out["e2e"] = {"value": bfly / (ms_e2e * 1e-3), "unit": "butterflies/s", "ms_per_step": ms_e2e,
                  "h2d_bytes_per_step": host_in.numel() * 8, "d2h_bytes_per_step": host_out[0].numel() * 8,
                  "bit_exact": bool(exact), "steps": n_e2e, "jobs": E2E_JOBS,
                  "form": f"pipelined: later steps' input copies and earlier steps' result copies overlap each "
                          f"step ({nbuf} device buffers, two copy streams); value = steps / total time of a job, "
                          f"median of {E2E_JOBS} jobs",
                  "link_ms_per_step": ms_link, "link_frac": ms_link / ms_e2e,
                  "serial_ms_per_step": ms_ser, "serial_value": bfly / (ms_ser * 1e-3)}
    del dbuf[1:], pbs[1:]

    if not args.no_blas:
        progress("BLAS")
        out["blas"] = bench_blas(M, torch, dev, stream, flush)
        out["small_ntt"] = bench_small_ntt(M, torch, dev, stream)
    if not args.no_other_width:
        progress("uniform batch at the other width")
        out["c3_other_width"] = bench_c3_width(M, torch, dev, stream, flush, args, 60 if args.bits == 124 else 124)
    if not args.no_uneven:
        progress("uneven batch")
        mix = uneven_mix(M, torch, dev)
        out["uneven"] = bench_uneven(M, torch, dev, stream, flush, args.steps, batch_opts(M, args), mix)
        if not args.no_serve:
            progress("serving sweep")
            out["serve"] = serve_sweep(M, torch, mix, args.serve_point_seconds)
        del mix
    if width == 2:   # the two forms of the double-word product (Sec. 2.2, Eq. 8 and 9), multiply-bound
        r_s, _ = M.mq_probe_mulmod_rate(M.MQ_MUL_SCHOOLBOOK, 2000, q, stream=sh)
        r_k, _ = M.mq_probe_mulmod_rate(M.MQ_MUL_KARATSUBA, 2000, q, stream=sh)
        out["product_forms"] = {"what": "general 124-bit modular products (Barrett) per second on register-resident "
                                        "operands, schoolbook vs Karatsuba double-word product",
                                "schoolbook_mulmod_per_s": r_s, "karatsuba_mulmod_per_s": r_k,
                                "karatsuba_over_schoolbook": r_k / r_s}
    if not args.no_wide:
        progress("wide residues")
        out["wide"] = bench_wide(M, torch, dev, sh, timed, args)
    if not args.no_polymul:
        progress("polynomial product")
        out["polymul"] = bench_polymul(M, torch, dev, sh, timed, plan, d, batch, N, q, width, wl, mads_per_mul,
                                       alu_peak, args)

    out["clocks"] = clocks
    return out


def bench_c3_width(M, torch, dev, stream, flush, args, bits):
    """The uniform batch at another residue width (C3's second prime): per step, the batched
    persistent form, one call per direction over the batch, and one call per polynomial and
    direction; median event time with L2 flushed between steps; round trip and sampled forward
    outputs checked."""
    a2 = argparse.Namespace(**vars(args))
    a2.bits = bits
    wl = workload(a2)
    from paper_2509_12494_gb300 import workload as W
    N, batch, width = wl["N"], wl["batch"], wl["width"]
    sh = stream.cuda_stream
    flags = M.MQ_ORDER_BITREV if args.order == "bitrev" else M.MQ_ORDER_NATURAL
    plan = M.ntt_plan_create(wl["log2n"], wl["q"], wl["psi"], width, flags, stream=sh)
    x = W.gen_residues(batch * N, wl["q"], seed=12, width=width)
    d = M.to_device(x, dev)
    jobs = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, plan, d[b * N:(b + 1) * N], 1, N) for b in range(batch)]
    jobs += [M.ntt_job(M.MQ_JOB_NTT_INVERSE, plan, d[b * N:(b + 1) * N], 1, N, after=b) for b in range(batch)]
    pb = M.mq_batch_create(jobs, batch_opts(M, args), stream=sh)

    def batched():
        M.mq_batch_launch(pb, stream=sh)

    def call():
        M.ntt_forward(plan, d, batch, N, stream=sh)
        M.ntt_inverse(plan, d, batch, N, stream=sh)

    def plain():
        for b in range(batch):
            M.ntt_forward(plan, d[b * N:(b + 1) * N], 1, N, stream=sh)
        for b in range(batch):
            M.ntt_inverse(plan, d[b * N:(b + 1) * N], 1, N, stream=sh)

    reps = max(5, args.steps)
    ms_b, _ = time_reps(torch, stream, batched, flush, reps, args.warmup)
    ok = M.mq_batch_status(pb) == 0
    ms_c, _ = time_reps(torch, stream, call, flush, reps, 2)
    ms_p, _ = time_reps(torch, stream, plain, flush, max(3, reps // 3), 1)
    torch.cuda.synchronize()
    ok = ok and bool(np.array_equal(M.to_host(d), x))
    fwd_ok, fwd_n, fwd_call = check_forward_samples(M, torch, dev, sh, plan, x, wl, args.order == "bitrev",
                                                    batch_opts(M, args))
    bfly = 2 * wl["butterflies_per_dir"]
    del pb, d
    return {"workload": workload_name(wl, a2), "q_bits": bits, "ms_batched": ms_b, "ms_call": ms_c, "ms_plain": ms_p,
            "butterflies_per_s": bfly / (ms_b * 1e-3), "call_butterflies_per_s": bfly / (ms_c * 1e-3),
            "plain_butterflies_per_s": bfly / (ms_p * 1e-3), "roundtrip_bit_exact": ok,
            "forward_sampled_bit_exact": fwd_ok and fwd_call, "forward_samples": fwd_n}


def bench_wide(M, torch, dev, sh, timed, args):
    """Residues of three and four 64-bit words (192- and 256-bit q, the larger bit-widths of Sec. 7):
    forward + inverse transform of 64 polynomials of N = 2^16, one call per direction, bit-exact
    round trip checked."""
    from paper_2509_12494_gb300 import workload as W
    res = {}
    batch, log2n = 64, 16
    N = 1 << log2n
    for width, bits in ((3, 188), (4, 252)):
        q = W.gen_prime(bits, 18, 1)
        plan = M.ntt_plan_create(log2n, q, W.gen_root(q, log2n, 1), width, M.MQ_ORDER_BITREV, stream=sh)
        d = M.to_device(W.gen_residues(batch * N, q, seed=width, width=width), dev)
        x0 = d.clone()

        def step():
            M.ntt_forward(plan, d, batch, N, stream=sh)
            M.ntt_inverse(plan, d, batch, N, stream=sh)

        ms = statistics.median(timed(step, args.steps, args.warmup))
        torch.cuda.synchronize()
        bfly = 2 * batch * (N // 2) * log2n
        res[f"w{64 * width}"] = {"q_bits": bits, "ms_per_step": ms, "butterflies_per_s": bfly / (ms * 1e-3),
                                 "roundtrip_bit_exact": bool(torch.equal(d, x0))}
        del d, x0, plan
    res["workload"] = f"{batch} x N=2^{log2n} negacyclic forward+inverse per width, bit-reversed order"
    return res


def bench_polymul(M, torch, dev, sh, timed, plan, d, batch, N, q, width, wl, mads_per_mul, alu_peak, args):
    """The batch's polynomial products c_i = a_i * b_i mod (x^N + 1): ntt_polymul (the product fused
    into the pass holding the last forward and first inverse stages) against the unfused sequence
    ntt_forward(a), ntt_forward(b), mod_vmul, ntt_inverse on the same operands (on stream `sh`,
    the one `timed` records its events on)."""
    gen = torch.Generator(device=dev)
    gen.manual_seed(77)
    b = dev_residues(torch, batch * N, q, width, gen, dev).view_as(d)
    c = torch.empty_like(d)
    ta, tb = d.clone(), b.clone()
    # bit-exactness of what is timed: fused and unfused on the same inputs
    M.ntt_polymul(plan, c, d, b, batch, N, stream=sh)
    M.ntt_forward(plan, ta, batch, N, stream=sh)
    M.ntt_forward(plan, tb, batch, N, stream=sh)
    M.mod_vmul(ta, ta, tb, batch * N, q, width, stream=sh)
    M.ntt_inverse(plan, ta, batch, N, stream=sh)
    torch.cuda.synchronize()
    same = bool(torch.equal(c, ta))

    def step_fused():
        M.ntt_polymul(plan, c, d, b, batch, N, stream=sh)

    def step_unfused():   # in place on the copies: the arithmetic's cost does not depend on the values
        M.ntt_forward(plan, ta, batch, N, stream=sh)
        M.ntt_forward(plan, tb, batch, N, stream=sh)
        M.mod_vmul(ta, ta, tb, batch * N, q, width, stream=sh)
        M.ntt_inverse(plan, ta, batch, N, stream=sh)

    ms_f = statistics.median(timed(step_fused, args.steps, args.warmup))
    ms_u = statistics.median(timed(step_unfused, args.steps, args.warmup))
    barrett_mads = MADS_PER_BARRETT[width]   # 32-bit multiply instructions per Barrett product
    mads = (3 * wl["butterflies_per_dir"] + batch * N // 2) * mads_per_mul + batch * N * barrett_mads
    del b, c, ta, tb
    return {"workload": f"{batch} products of degree-{N} polynomials mod (x^N + 1), {q.bit_length()}-bit q",
            "products_per_s": batch / (ms_f * 1e-3), "ms_fused": ms_f, "ms_unfused": ms_u,
            "fused_over_unfused": ms_u / ms_f, "bit_exact_vs_unfused": same,
            "launches_fused": 1 if N <= 4096 else 4, "launches_unfused": (1 if N <= 4096 else 2) * 3 + 1,
            "alu_frac": mads / (ms_f * 1e-3) / alu_peak,
            "alu_count": f"3 transforms x {mads_per_mul} per butterfly + N/2 scale products + N Barrett products "
                         f"x {barrett_mads} (32-bit multiply instructions)"}


def time_reps(torch, stream, call, flush=None, reps=20, warm=5):
    """Median and min event time (ms) of `call` over `reps` timed reps after `warm` untimed ones; the L2
    flush (if given) runs between reps, outside the events."""
    times = []
    with torch.cuda.stream(stream):
        for i in range(warm + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            if flush is not None:
                flush_l2(flush)
            if i >= warm:
                times.append((e0, e1))
        torch.cuda.synchronize()
    ms = [x.elapsed_time(y) for x, y in times]
    return statistics.median(ms), min(ms)


def back_to_back(torch, stream, call, k=20):
    """Mean event time (ms) of `call` over k calls queued back to back on `stream` after one warm-up."""
    with torch.cuda.stream(stream):
        call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def bench_blas(M, torch, dev, stream, flush):
    """vadd / vsub / vmul / axpy, 60- and 124-bit q: n = 2^24 and 2^20 with L2 flushed between reps
    (2^20 also L2-warm), and the paper's n = 1024 (L2-warm, launch-latency bound)."""
    from paper_2509_12494_gb300 import workload as W
    res = {}
    sh = stream.cuda_stream
    hbm_peak = measured_peaks().get("hbm_gbs") or HBM_FALLBACK_GBS
    for bits, width in ((60, 1), (124, 2)):
        q = W.gen_prime(bits, 18, 2)
        s = 0x1234567 % q
        for log2n in (24, 20, 10):
            n = 1 << log2n
            a, b = M.to_device(W.gen_residues(n, q, 1, width), dev), M.to_device(W.gen_residues(n, q, 2, width), dev)
            c = torch.empty_like(a)
            for op in ("vadd", "vsub", "vmul", "axpy"):
                def call():
                    if op == "axpy":
                        M.mod_axpy(c, s, a, n, q, width, stream=sh)
                    else:
                        getattr(M, "mod_" + op)(c, a, b, n, q, width, stream=sh)
                nbytes = 3 * n * 8 * width
                if log2n == 10:
                    ms, ms_min = time_reps(torch, stream, call)
                    entry = {"us": ms * 1e3, "us_min": ms_min * 1e3, "elements/s": n / (ms * 1e-3),
                             "l2": "warm (the 48 KiB working set stays on chip)"}
                else:
                    ms, ms_min = time_reps(torch, stream, call, flush)
                    gbs = nbytes / (ms * 1e-3) / 1e9
                    entry = {"ms": ms, "ms_min": ms_min, "GB/s": gbs, "hbm_frac": gbs / hbm_peak,
                             "elements/s": n / (ms * 1e-3)}
                    if log2n == 20:
                        ms_w, _ = time_reps(torch, stream, call)
                        entry["ms_l2_warm"] = ms_w
                        entry["GB/s_l2_warm"] = nbytes / (ms_w * 1e-3) / 1e9
                        # device time without the host's call latency: 20 launches back to back between
                        # two events (each followed by the L2 flush, whose own time is subtracted)
                        ms_fl = back_to_back(torch, stream, lambda: flush_l2(flush))
                        ms_d = back_to_back(torch, stream, lambda: (call(), flush_l2(flush))) - ms_fl
                        entry["ms_device"] = ms_d
                        entry["GB/s_device"] = nbytes / (ms_d * 1e-3) / 1e9
                        entry["ms_device_l2_warm"] = back_to_back(torch, stream, call)
                if op in ("vmul", "axpy"):
                    entry["modmul/s"] = entry["elements/s"]
                res[f"{op}_{bits}" if log2n == 24 else f"{op}_{bits}_n2^{log2n}"] = entry
            del a, b, c
    return res


def bench_small_ntt(M, torch, dev, stream):
    """One negacyclic forward + inverse transform of N = 1024 under a 124-bit q = 1 mod 2048 (seeds 1..5),
    as two calls and as a two-job batch replayed from a graph: latency-bound (one CTA), L2-warm."""
    from paper_2509_12494_gb300 import workload as W
    sh = stream.cuda_stream
    log2n, N = 10, 1024
    bfly = 2 * (N // 2) * log2n
    per_seed = []
    exact = True
    for seed in range(1, 6):
        q = W.gen_prime(124, log2n + 1, seed)
        psi = W.gen_root(q, log2n, seed)
        plan = M.ntt_plan_create(log2n, q, psi, 2, 0, stream=sh)
        x = W.gen_residues(N, q, seed, 2)
        d = M.to_device(x, dev)

        def calls():
            M.ntt_forward(plan, d, 1, N, stream=sh)
            M.ntt_inverse(plan, d, 1, N, stream=sh)
        jobs = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, plan, d, 1, N), M.ntt_job(M.MQ_JOB_NTT_INVERSE, plan, d, 1, N, after=0)]
        pb = M.mq_batch_create(jobs, None, stream=sh)

        def graph():
            M.mq_batch_launch(pb, stream=sh)
        ms_c, min_c = time_reps(torch, stream, calls)
        ms_g, min_g = time_reps(torch, stream, graph)
        exact = exact and bool(np.array_equal(M.to_host(d), x)) and M.mq_batch_status(pb) == 0
        per_seed.append((ms_c, min_c, ms_g, min_g))
        del pb
    med = lambda k: statistics.median(r[k] for r in per_seed)
    return {"workload": "1 x N=1024 negacyclic forward+inverse, 124-bit q = 1 mod 2048, seeds 1..5, "
                        "median over seeds of the median of 20 reps",
            "butterflies": bfly, "roundtrip_bit_exact": exact,
            "calls_us": med(0) * 1e3, "calls_us_min": min(r[1] for r in per_seed) * 1e3,
            "calls_butterflies/s": bfly / (med(0) * 1e-3),
            "graph_us": med(2) * 1e3, "graph_us_min": min(r[3] for r in per_seed) * 1e3,
            "graph_butterflies/s": bfly / (med(2) * 1e-3)}


# ----------------------------------------------------------------------------------- uneven batch

def dev_residues(torch, n, q, width, gen, dev):
    """n residues uniform in [0, q) generated on the device (rejection on bitlen(q)-bit draws)."""
    bits = q.bit_length()

    def draw64(m):
        a = torch.empty(m, dtype=torch.int64, device=dev).random_(generator=gen)
        b = torch.empty(m, dtype=torch.int64, device=dev).random_(generator=gen)
        return (a & 0xFFFFFFFF) | (b << 32)

    if width == 1:
        mask = (1 << bits) - 1
        x = draw64(n) & mask
        while True:
            bad = x >= q
            k = int(bad.sum())
            if k == 0:
                return x
            x[bad] = draw64(k) & mask
    qlo, qhi = q & (2**64 - 1), q >> 64
    sign = -(2**63)
    qlo_s = (qlo ^ (1 << 63)) - (1 << 64) if (qlo ^ (1 << 63)) >= (1 << 63) else (qlo ^ (1 << 63))
    hmask = (1 << (bits - 64)) - 1
    out = torch.empty((n, 2), dtype=torch.int64, device=dev)
    lo, hi = draw64(n), draw64(n) & hmask
    while True:
        lo_s = lo ^ sign
        bad = (hi > qhi) | ((hi == qhi) & (lo_s >= qlo_s))
        k = int(bad.sum())
        if k == 0:
            break
        lo[bad] = draw64(k)
        hi[bad] = draw64(k) & hmask
    out[:, 0], out[:, 1] = lo, hi
    return out


def uneven_mix(M, torch, dev, seed=4):
    """512 transforms (N uniform over 2^12..2^17, 60- or 124-bit prime q = 1 mod 2^18 of their own,
    forward then inverse) interleaved with 512 BLAS jobs (vmul or axpy, length 2^k with k uniform
    in 14..22, 60- or 124-bit).  Returns jobs for the batch form and work counts."""
    from paper_2509_12494_gb300 import workload as W
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    ntt, blas = [], []
    for i in range(512):
        log2n = int(rng.integers(12, 18))
        bits = int(rng.choice([60, 124]))
        width = 2 if bits > 60 else 1
        q = W.gen_prime(bits, 18, 10000 + i)
        psi = W.gen_root(q, log2n, i)
        plan = M.ntt_plan_create(log2n, q, psi, width, M.MQ_ORDER_BITREV)
        d = dev_residues(torch, 1 << log2n, q, width, gen, dev)
        ntt.append(dict(plan=plan, d=d, N=1 << log2n, log2n=log2n))
    for i in range(512):
        k = int(rng.integers(14, 23))
        bits = int(rng.choice([60, 124]))
        width = 2 if bits > 60 else 1
        q = W.gen_prime(bits, 18, 20000 + i)
        n = 1 << k
        op = "vmul" if rng.integers(0, 2) == 0 else "axpy"
        a = dev_residues(torch, n, q, width, gen, dev)
        b = dev_residues(torch, n, q, width, gen, dev)
        c = torch.empty_like(a) if op == "vmul" else b
        s = int(rng.integers(1, 2**62)) % q
        blas.append(dict(op=op, a=a, b=b, c=c, n=n, q=q, width=width, s=s))
    jobs = []
    for i in range(512):   # interleaved: forward i, its inverse, BLAS i
        t = ntt[i]
        jobs.append(M.ntt_job(M.MQ_JOB_NTT_FORWARD, t["plan"], t["d"], 1, t["N"]))
        jobs.append(M.ntt_job(M.MQ_JOB_NTT_INVERSE, t["plan"], t["d"], 1, t["N"], after=len(jobs) - 1))
        bj = blas[i]
        kind = M.MQ_JOB_VMUL if bj["op"] == "vmul" else M.MQ_JOB_AXPY
        jobs.append(M.blas_job(kind, bj["c"], bj["a"], bj["b"], bj["n"], bj["q"], bj["width"], bj["s"]))
    bfly = sum(2 * (t["N"] // 2) * t["log2n"] for t in ntt)
    mm = sum(b["n"] for b in blas)
    return dict(ntt=ntt, blas=blas, jobs=jobs, butterflies=bfly, blas_modmuls=mm)


def describe_opts(M, o):
    """The options a batch was built with, for the report."""
    form = ("calls" if o.flags & M.MQ_BATCH_FORM_CALLS else "split" if o.flags & M.MQ_BATCH_FORM_SPLIT
            else "prefetch")
    return {"form": form, "ctas_per_sm": o.ctas_per_sm, "lag": o.lag, "blas_chunk": o.blas_chunk,
            "split_shift": o.split_shift}


def batch_opts(M, args):
    """Options of the persistent batches from the command line (None: the library's defaults)."""
    form_flag = {"default": 0, "split": M.MQ_BATCH_FORM_SPLIT, "prefetch": M.MQ_BATCH_FORM_PREFETCH}[args.form]
    if not (args.lag or args.ctas_per_sm or form_flag):
        return None
    return M.mq_batch_opts(lag=args.lag, ctas_per_sm=args.ctas_per_sm, flags=form_flag)


def bench_uneven(M, torch, dev, stream, flush, steps, opts=None, mix=None, tune=True):
    mix = mix or uneven_mix(M, torch, dev)
    sh = stream.cuda_stream
    # every job's inputs as they were: NTT data (transformed in place) and axpy's y (updated in place)
    saved_ntt = [t["d"].clone() for t in mix["ntt"]]
    saved_y = [bj["c"].clone() if bj["op"] == "axpy" else None for bj in mix["blas"]]
    tuned = None
    if opts is None and tune:
        # the library's autotuner on this batch shape (it runs the batch, so the inputs are restored
        # below); its choice goes through a cache file as a user's would
        import tempfile
        t0 = time.perf_counter()
        with tempfile.TemporaryDirectory() as tdir:
            progress("autotuning the uneven batch")
        opts = M.mq_autotune_batch(mix["jobs"], os.path.join(tdir, "tune.json"), stream=sh)
        progress("autotuned")
        tuned = describe_opts(M, opts)
        tuned["tune_s"] = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            for t, x0 in zip(mix["ntt"], saved_ntt):
                t["d"].copy_(x0)
            for bj, y0 in zip(mix["blas"], saved_y):
                if y0 is not None:
                    bj["c"].copy_(y0)
        torch.cuda.synchronize()
    b = M.mq_batch_create(mix["jobs"], opts, stream=sh)
    info = M.mq_batch_info(b)

    def step_batch():
        M.mq_batch_launch(b, stream=sh)

    def calls(inverse=True):
        for t, bj in zip(mix["ntt"], mix["blas"]):
            M.ntt_forward(t["plan"], t["d"], 1, t["N"], stream=sh)
            if inverse:
                M.ntt_inverse(t["plan"], t["d"], 1, t["N"], stream=sh)
            if bj["op"] == "vmul":
                M.mod_vmul(bj["c"], bj["a"], bj["b"], bj["n"], bj["q"], bj["width"], stream=sh)
            else:
                M.mod_axpy(bj["c"], bj["s"], bj["a"], bj["n"], bj["q"], bj["width"], stream=sh)

    def step_calls():
        calls(True)

    def timeit(step, k):
        with torch.cuda.stream(stream):
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            ts = []
            for _ in range(k):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                flush_l2(flush)
                ts.append((e0, e1))
            torch.cuda.synchronize()
        return statistics.median([x.elapsed_time(y) for x, y in ts])

    ms_b = timeit(step_batch, max(3, steps))
    status = M.mq_batch_status(b)
    progress(f"uneven batch timed ({ms_b:.2f} ms, status {status}); per-call path")
    ms_c = timeit(step_calls, max(2, steps // 2))
    progress("uneven batch: per-job checks")

    # checks of what was timed, job by job against the per-call path (itself pinned to the oracle
    # by the tests): (1) the timed batch once on the saved inputs; (2) the forward transforms and
    # the BLAS jobs as a batch of their own, so that the transforms' forward results are compared too
    def restore():
        for t, x0 in zip(mix["ntt"], saved_ntt):
            t["d"].copy_(x0)
        for bj, y0 in zip(mix["blas"], saved_y):
            if y0 is not None:
                bj["c"].copy_(y0)

    def outputs():
        return [t["d"].clone() for t in mix["ntt"]] + [bj["c"].clone() for bj in mix["blas"]]

    def same(xs, ys):
        return [bool(torch.equal(x, y)) for x, y in zip(xs, ys)]

    with torch.cuda.stream(stream):
        restore()
        step_batch()
        torch.cuda.synchronize()
        st1 = M.mq_batch_status(b)
        got = outputs()
        restore()
        calls(True)
        torch.cuda.synchronize()
        eq_all = same(got, outputs())
        roundtrip = all(torch.equal(t["d"], x0) for t, x0 in zip(mix["ntt"], saved_ntt))
        del got
        restore()
        fjobs = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, t["plan"], t["d"], 1, t["N"]) for t in mix["ntt"]]
        for bj in mix["blas"]:
            kind = M.MQ_JOB_VMUL if bj["op"] == "vmul" else M.MQ_JOB_AXPY
            fjobs.append(M.blas_job(kind, bj["c"], bj["a"], bj["b"], bj["n"], bj["q"], bj["width"], bj["s"]))
        fb = M.mq_batch_create(fjobs, opts, stream=sh)
        M.mq_batch_launch(fb, stream=sh)
        st2 = M.mq_batch_status(fb)
        got = outputs()
        restore()
        calls(False)
        torch.cuda.synchronize()
        eq_fwd = same(got, outputs())
        del got, fb
        restore()
        torch.cuda.synchronize()
    del saved_ntt, saved_y
    total = mix["butterflies"] + mix["blas_modmuls"]
    return {"workload": "uneven batch: 512 negacyclic NTTs (N uniform 2^12..2^17, own 60/124-bit prime each, "
                        "forward then inverse, bit-reversed order) interleaved with 512 vmul/axpy jobs "
                        "(length 2^14..2^22, 60/124-bit)",
            "modmul_per_s": total / (ms_b * 1e-3), "butterflies_per_s": mix["butterflies"] / (ms_b * 1e-3),
            "blas_modmul_per_s": mix["blas_modmuls"] / (ms_b * 1e-3), "ms_per_step": ms_b, "status": status,
            "items": info["items"], "per_call": {"modmul_per_s": total / (ms_c * 1e-3), "ms_per_step": ms_c,
                                                 "launches": 512 + sum(2 * (1 if t["N"] <= 4096 else 2) for t in mix["ntt"])},
            "batched_over_per_call": ms_c / ms_b, "butterflies": mix["butterflies"],
            "blas_modmuls": mix["blas_modmuls"],
            "autotuned": tuned,
            "jobs_bit_exact_vs_per_call": bool(all(eq_all) and st1 == 0 and roundtrip),
            "forward_jobs_bit_exact_vs_per_call": bool(all(eq_fwd) and st2 == 0),
            "jobs_checked": len(eq_all) + len(eq_fwd)}


def serve_sweep(M, torch, mix, seconds=0.5, fracs=(0.5, 1.0, 1.25)):
    """A short serving sweep on the uneven mix's jobs (single forward transforms and BLAS requests,
    Poisson arrivals): saturated throughput of both modes (everything submitted at once), then the
    given fractions of the batched mode's saturation, for both modes."""
    pool = [M.ntt_job(M.MQ_JOB_NTT_FORWARD, t["plan"], t["d"], 1, t["N"]) for t in mix["ntt"]]
    for bj in mix["blas"]:
        kind = M.MQ_JOB_VMUL if bj["op"] == "vmul" else M.MQ_JOB_AXPY
        pool.append(M.blas_job(kind, bj["c"], bj["a"], bj["b"], bj["n"], bj["q"], bj["width"], bj["s"]))
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    pool = [pool[i] for i in rng.permutation(len(pool))]

    def run(mode, rate, n_req, seed):
        srv = M.mq_server_create(M.mq_server_cfg(mode=mode))
        offered = M.mq_server_poisson(srv, pool, rate, n_req, seed)
        M.mq_server_drain(srv, 300)
        st = M.mq_server_stats(srv)
        M.mq_server_destroy(srv)
        return offered, st

    modes = (("batched", M.MQ_SERVE_BATCHED), ("plain", M.MQ_SERVE_PLAIN))
    sat = {name: run(mode, 0.0, 4 * len(pool), 1)[1]["jobs_per_s"] for name, mode in modes}
    progress(f"saturation {sat}")
    # the batched mode at fractions of its saturated rate; the plain mode at fractions of its own, and
    # at half the batched mode's saturated rate (far beyond what it sustains)
    plan = [("batched", M.MQ_SERVE_BATCHED, "batched", f) for f in fracs]
    plan += [("plain", M.MQ_SERVE_PLAIN, "plain", f) for f in (0.5, 1.0)]
    plan += [("plain", M.MQ_SERVE_PLAIN, "batched", 0.5)]
    points = []
    for name, mode, base, frac in plan:
        rate = frac * sat[base]
        n_req = int(max(200, min(rate * seconds, 200000)))
        offered, st = run(mode, rate, n_req, 7)
        progress(f"serving point {name} at {frac} x {base}: p50 {st['p50_ms']:.3f} ms")
        points.append({"mode": name, "load": frac, "of": base, "offered_per_s": offered, "jobs_per_s": st["jobs_per_s"],
                       "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "modmul_per_s": st["modmul_per_s"],
                       "failed": st["failed"]})
    return {"workload": "Poisson arrivals of single requests from the uneven mix (forward NTT 2^12..2^17 or "
                        "vmul/axpy 2^14..2^22, 60/124-bit), twiddles and operands resident, admission by free HBM; "
                        f"load = fraction of the saturated rate of mode `of`, {seconds} s of arrivals per point",
            "saturated_jobs_per_s": sat, "points": points}


# ----------------------------------------------------------------------------------- serving

def run_serve(args):
    """Open-loop Poisson arrivals of single requests drawn from the uneven mix (a forward or an
    inverse transform, or a BLAS job), at a geometric sweep of rates, through the batching server
    and through the plain per-call mode.  A request's buffers are not reused while it is in flight
    (a busy buffer delays that arrival, which only happens near saturation)."""
    import torch

    from paper_2509_12494_gb300 import mqntt as M
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    M.load(build_if_missing=True)
    mix = uneven_mix(M, torch, dev, seed=5)
    pool = []
    for t in mix["ntt"]:
        pool.append(M.ntt_job(M.MQ_JOB_NTT_FORWARD, t["plan"], t["d"], 1, t["N"]))
    for bj in mix["blas"]:
        kind = M.MQ_JOB_VMUL if bj["op"] == "vmul" else M.MQ_JOB_AXPY
        pool.append(M.blas_job(kind, bj["c"], bj["a"], bj["b"], bj["n"], bj["q"], bj["width"], bj["s"]))
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    pool = [pool[i] for i in rng.permutation(len(pool))]
    out = {"metric": METRIC, "impl": "mq", "workload": "serve", "unit": "requests/s",
           "config": {"workload": "serving: Poisson arrivals of single NTT (2^12..2^17, 60/124-bit) and "
                                  "vmul/axpy (2^14..2^22) requests, twiddles and operands resident, "
                                  "admission by free HBM", "seconds_per_rate": args.serve_seconds},
           "points": []}

    def run(mode, rate, n_req, seed):
        srv = M.mq_server_create(M.mq_server_cfg(mode=mode))
        offered = M.mq_server_poisson(srv, pool, rate, n_req, seed)
        M.mq_server_drain(srv, 300)
        st = M.mq_server_stats(srv)
        M.mq_server_destroy(srv)
        return offered, st

    # saturated throughput of each mode: everything submitted at once
    sat = {}
    for mode_name, mode in (("batched", M.MQ_SERVE_BATCHED), ("plain", M.MQ_SERVE_PLAIN)):
        _, st = run(mode, 0.0, 4 * len(pool), 1)
        sat[mode_name] = st["jobs_per_s"]
    out["saturated_jobs_per_s"] = sat
    base = sat["batched"]
    for mode_name, mode in (("batched", M.MQ_SERVE_BATCHED), ("plain", M.MQ_SERVE_PLAIN)):
        for frac in (0.1, 0.2, 0.35, 0.5, 0.7, 0.85, 1.0, 1.25, 1.5):
            rate = frac * base
            n_req = int(max(200, min(rate * args.serve_seconds, 200000)))
            offered, st = run(mode, rate, n_req, 7)
            out["points"].append({"mode": mode_name, "rate_frac_of_batched_saturation": frac, "rate": rate,
                                  "offered_per_s": offered, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                                  "jobs_per_s": st["jobs_per_s"], "modmul_per_s": st["modmul_per_s"],
                                  "butterflies_per_s": st["butterflies_per_s"],
                                  "mean_batch_jobs": st["mean_batch_jobs"], "failed": st["failed"]})
    return out


# ----------------------------------------------------------------------------------- oracle arms

def oracle_sample(args, wl, n_jobs, which="both"):
    """Time the oracle on n_jobs of the workload's transforms on all host cores; butterflies/s."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2509_12494_gb300 import workload as W
    cores = os.cpu_count() or 1
    O = oracle.default()
    xs = [W.gen_residues(wl["N"], wl["q"], seed=100 + i, width=wl["width"]) for i in range(n_jobs)]
    flags = oracle.BITREV if args.order == "bitrev" else 0

    def job(i):
        inverse = (which == "inverse") or (which == "both" and i % 2 == 1)
        O.ntt(xs[i], wl["log2n"], wl["q"], wl["psi"], wl["width"], flags, inverse=inverse)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(job, range(n_jobs)))
    dt = time.perf_counter() - t0
    bfly = n_jobs * (wl["N"] // 2) * wl["log2n"]
    return bfly / dt, dt, cores


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload(args)
    cores = os.cpu_count() or 1
    n_jobs = cores
    for _ in range(args.warmup):
        oracle_sample(args, wl, max(1, cores // 4))
    times = []
    for _ in range(args.steps):
        v, dt, _ = oracle_sample(args, wl, n_jobs)
        times.append(dt)
    dt = sum(times) / len(times)
    bfly = n_jobs * (wl["N"] // 2) * wl["log2n"]
    value = bfly / dt
    sample = (f"{n_jobs} of the {wl['batch']} transforms per step (half forward, half inverse), "
              f"one per host thread")
    return {"metric": METRIC, "value": value, "unit": "butterflies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u128" if wl["width"] == 2 else "u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(wl, args), "batch": wl["batch"], "log2n": wl["log2n"],
                       "q_bits": args.bits, "order": args.order},
            "cpu_baseline": {"value": value, "unit": "butterflies/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "butterflies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_int8_probe(args):
    """The tensor-core question for a limb-split NTT stage: the dense int8 GEMM rate of this GPU
    (cuBLASLt through torch._int_mm, int8 x int8 -> int32), and the butterfly rate that rate would
    bound a limb-split radix-16 stage to.  A 16-point transform over Z_q as a dense 16 x 16 product
    on 8-bit limbs of 124-bit residues takes 16 x 16 limb pairs per coefficient product and 16 x 16
    coefficient products per 16 outputs, which stand for 4 radix-2 stages of 8 butterflies: 2048
    multiply-adds (4096 int8 operations) per butterfly, before the reductions mod q of the wide
    accumulators, which run on the CUDA cores on top."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def rate(n, dtype):
        if dtype == torch.int8:
            a = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev)
            b = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev)
            mm = torch._int_mm
        else:
            a = torch.randint(0, 256, (n, n), device=dev).to(dtype)
            b = torch.randint(0, 256, (n, n), device=dev).to(dtype)
            mm = torch.matmul
        for _ in range(3):
            mm(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        return 2 * n ** 3 / (e0.elapsed_time(e1) / reps * 1e-3)

    rates = {n: rate(n, torch.int8) for n in args.int8_n}
    bf16 = {n: rate(n, torch.bfloat16) for n in args.int8_n}
    ops = max(rates.values())
    per_bfly = 2 * 16 * 16 * 16 * 16 / 32
    # the exact bf16 formulation: K = 16 inputs x 16 limbs of 8 bits (partial sums below 2^24, exact
    # in fp32), a Toeplitz-expanded operand of 31 limb shifts per column, 16 outputs per 32 butterflies
    bf16_per_bfly = 2 * 16 * 256 * 31 / 32
    return {"metric": METRIC, "workload": "int8-probe", "int8_ops_per_s": ops,
            "by_size": {str(k): v for k, v in rates.items()},
            "bf16_ops_per_s": max(bf16.values()), "bf16_by_size": {str(k): v for k, v in bf16.items()},
            "limb_split_int8_ops_per_butterfly": per_bfly,
            "butterfly_bound_per_s": ops / per_bfly,
            "bf16_limb_split_flops_per_butterfly": bf16_per_bfly,
            "bf16_butterfly_bound_per_s": max(bf16.values()) / bf16_per_bfly,
            "note": "upper bound from the tensor part alone; the reductions mod q of the wide accumulators "
                    "(CUDA cores) come on top"}


def _r(v, nd=4):
    """Round to nd significant digits (compact summary numbers)."""
    if v is None or isinstance(v, bool):
        return v
    return float(f"{v:.{nd}g}")


def tail_summary(out):
    """Every config's headline numbers, compact, as the last key of the line (the part of the line a
    reader sees first when only its end is kept).  Moves itself to the end."""
    s = {"c3": {"bits": out["config"]["q_bits"], "ms_batched": _r(out["ms_per_step"]),
                "ms_call": _r(out.get("batched_call", {}).get("ms_per_step")),
                "ms_plain": _r(out.get("plain", {}).get("ms_per_step")),
                "ms_e2e": _r(out.get("e2e", {}).get("ms_per_step")),
                "fwd_exact": out.get("forward_sampled_bit_exact"), "rt_exact": out.get("roundtrip_bit_exact"),
                "alu_frac": _r(out.get("roofline", {}).get("frac"), 3)}}
    o = out.get("c3_other_width")
    if o:
        s["c3_other"] = {"bits": o["q_bits"], "ms_batched": _r(o["ms_batched"]), "ms_call": _r(o["ms_call"]),
                         "ms_plain": _r(o["ms_plain"]), "exact": o["roundtrip_bit_exact"] and o["forward_sampled_bit_exact"]}
    u = out.get("uneven")
    if u:
        s["c4"] = {"ms_batched": _r(u["ms_per_step"]), "ms_per_call": _r(u["per_call"]["ms_per_step"]),
                   "modmul_per_s": _r(u["modmul_per_s"]), "exact": u["jobs_bit_exact_vs_per_call"] and
                   u["forward_jobs_bit_exact_vs_per_call"],
                   "tuned": ({k: v for k, v in u["autotuned"].items() if k != "tune_s"} if u.get("autotuned") else None)}
    v = out.get("serve")
    if v:
        s["c5"] = {"sat_jobs_per_s": {k: _r(x, 3) for k, x in v["saturated_jobs_per_s"].items()},
                   "p50_p99_ms_jobs_per_s": {f"{p['mode']}@{p['load']}x{p['of'][0]}": [_r(p["p50_ms"], 3), _r(p["p99_ms"], 3),
                                                                                        _r(p["jobs_per_s"], 3)]
                                             for p in v["points"]}}
    b = out.get("blas")
    if b:
        s["c2_GBps"] = {k: _r(b[k].get("GB/s"), 3) for k in ("vadd_124", "vmul_124", "axpy_124", "vadd_60", "vmul_60")
                        if k in b}
        s["c2_GBps"]["vadd_124_2^20_dev"] = _r(b.get("vadd_124_n2^20", {}).get("GB/s_device"), 3)
        s["c2_GBps"]["vmul_124_2^20_dev"] = _r(b.get("vmul_124_n2^20", {}).get("GB/s_device"), 3)
    n = out.get("small_ntt")
    if n:
        s["c1_us"] = {"calls": _r(n["calls_us"], 3), "graph": _r(n["graph_us"], 3), "exact": n["roundtrip_bit_exact"]}
    out.pop("summary", None)
    out["summary"] = s
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "serve":
        out = run_serve(args) if rank == 0 else None
    elif args.workload == "int8-probe":
        out = run_int8_probe(args) if rank == 0 else None
    else:
        out = run_gpu(args, rank, world)
        if out is not None and not args.no_cpu_baseline:
            progress("oracle on the host cores")
            wl = workload(args)
            cores = os.cpu_count() or 1
            v, dt, cores = oracle_sample(args, wl, cores)
            out["cpu_baseline"] = {"value": v, "unit": "butterflies/s", "cores": cores, "kind": "oracle",
                                   "sample": f"{cores} of the {wl['batch']} transforms (half forward, half "
                                             f"inverse), one per host thread, {dt:.1f} s wall"}
    if out is not None and rank == 0:
        if "ms_per_step" in out and "config" in out and args.impl != "reference":
            tail_summary(out)
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

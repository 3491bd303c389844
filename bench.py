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
    p.add_argument("--lag", type=int, default=0, help="pipeline lag of the persistent batch (0: library default)")
    p.add_argument("--ctas-per-sm", type=int, default=0, help="persistent CTAs per SM (0: library default)")
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
    opts = M.mq_batch_opts(lag=args.lag, ctas_per_sm=args.ctas_per_sm) if (args.lag or args.ctas_per_sm) else None
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

    def timed(step, steps, warmup, sampler_idx=None):
        """Per-step device time (ms) with CUDA events on the launching stream; L2 flushed between."""
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step()
                flush_l2(flush)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            times = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                flush_l2(flush)
                times.append((e0, e1))
            torch.cuda.synchronize()
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

    with ClockSampler(dev.index) as clk:
        t_batched = timed(step_batched, args.steps, args.warmup)
        clocks = clk.summary()
    ms = sum(t_batched) / len(t_batched)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    bfly = 2 * wl["butterflies_per_dir"]
    value = bfly * world / (ms * 1e-3)

    # correctness of what was timed: the round trip leaves the input unchanged
    batch_status = M.mq_batch_status(pbatch)
    ok_roundtrip = bool(np.array_equal(M.to_host(d), x_host)) and batch_status == 0

    out = {"metric": METRIC, "value": value, "unit": "butterflies/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u128" if width == 2 else "u64", "data": "synthetic",
           "config": {"workload": workload_name(wl, args), "batch": batch, "log2n": wl["log2n"],
                      "q_bits": args.bits, "order": args.order,
                      "form": f"batched persistent kernel in a CUDA graph ({pinfo['items']} work items, "
                              f"{pinfo['ctas']} CTAs)",
                      "l2": "L2 flushed between timed steps (2 x L2 write); working set "
                            f"{batch * N * 8 * width >> 20} MiB", "parallelism": f"replicas x{world}"},
           "roundtrip_bit_exact": ok_roundtrip}

    # gpu launches in the timed region: one persistent kernel per step (plus a counter memset and
    # a 4-byte status copy in the same graph)
    passes = 1 if wl["log2n"] <= 12 else 2
    out["gpu_launches"] = args.steps

    if rank != 0:
        return None

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
    mads_per_mul = 64 if width == 2 else 16   # 32-bit multiply instructions per Shoup product
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
    if alu_frac >= hbm_frac:
        out["roofline"] = {"bound": "alu", "achieved": alu_achieved / 1e12, "peak": alu_peak / 1e12,
                           "unit": "T mad32/s", "frac": alu_frac, "traffic": None,
                           "kernel": "persistent_kernel (one launch = one step)",
                           "peak_source": "measured by mq_probe_imad_rate (carry-chained mad.lo.cc/madc.hi.cc)",
                           "algorithmic": f"{mads_per_mul} 32-bit multiply instructions per Shoup product",
                           "hbm_frac": hbm_frac, "hbm_achieved_gbs": hbm_achieved,
                           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src, "ms_launch": ms_launch}
    else:
        out["roofline"] = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                           "frac": hbm_frac, "traffic": None, "kernel": "persistent_kernel (one launch = one step)",
                           "peak_source": hbm_src, "alu_frac": alu_frac, "ms_launch": ms_launch,
                           "alu_achieved_tmads": alu_achieved / 1e12, "alu_peak_tmads": alu_peak / 1e12}
    out["roofline"]["call_form_alu_frac"] = (mad_f + mad_i) / ((ms_f + ms_i) * 1e-3) / alu_peak
    out["roofline"]["call_form_ms_forward"] = ms_f
    out["roofline"]["call_form_ms_inverse"] = ms_i
    out["probe_mad_per_s"] = probe

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    host_in = torch.from_numpy(x_host.view(np.int64)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def step_e2e():
        d.copy_(host_in.view_as(d), non_blocking=True)
        step_batched()
        host_out.view_as(d).copy_(d, non_blocking=True)

    t_e2e = timed(step_e2e, max(3, args.steps // 2), 1)
    ms_e2e = sum(t_e2e) / len(t_e2e)
    torch.cuda.synchronize()
    out["e2e"] = {"value": bfly / (ms_e2e * 1e-3), "unit": "butterflies/s", "ms_per_step": ms_e2e,
                  "h2d_bytes_per_step": host_in.numel() * 8, "d2h_bytes_per_step": host_out.numel() * 8,
                  "bit_exact": bool(np.array_equal(host_out.numpy().view(np.uint64).reshape(x_host.shape), x_host))}

    if not args.no_blas:
        out["blas"] = bench_blas(M, torch, dev, stream, flush)

    out["clocks"] = clocks
    return out


def bench_blas(M, torch, dev, stream, flush):
    """vadd / vsub / vmul / axpy over n = 2^24 residues, 60- and 124-bit q, L2 flushed between reps."""
    from paper_2509_12494_gb300 import workload as W
    res = {}
    n = 1 << 24
    sh = stream.cuda_stream
    hbm_peak = measured_peaks().get("hbm_gbs") or HBM_FALLBACK_GBS
    for bits, width in ((60, 1), (124, 2)):
        q = W.gen_prime(bits, 18, 2)
        a, b = M.to_device(W.gen_residues(n, q, 1, width), dev), M.to_device(W.gen_residues(n, q, 2, width), dev)
        c = torch.empty_like(a)
        s = 0x1234567 % q
        for op in ("vadd", "vsub", "vmul", "axpy"):
            def call():
                if op == "axpy":
                    M.mod_axpy(c, s, a, n, q, width, stream=sh)
                else:
                    getattr(M, "mod_" + op)(c, a, b, n, q, width, stream=sh)
            times = []
            with torch.cuda.stream(stream):
                for i in range(13):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    call()
                    e1.record(stream)
                    flush_l2(flush)
                    if i >= 3:
                        times.append((e0, e1))
                torch.cuda.synchronize()
            ms = statistics.median([x.elapsed_time(y) for x, y in times])
            gbs = 3 * n * 8 * width / (ms * 1e-3) / 1e9
            entry = {"ms": ms, "GB/s": gbs, "hbm_frac": gbs / hbm_peak, "elements/s": n / (ms * 1e-3)}
            if op in ("vmul", "axpy"):
                entry["modmul/s"] = n / (ms * 1e-3)
            res[f"{op}_{bits}"] = entry
        del a, b, c
    return res


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
    else:
        out = run_gpu(args, rank, world)
        if out is not None and not args.no_cpu_baseline:
            wl = workload(args)
            cores = os.cpu_count() or 1
            v, dt, cores = oracle_sample(args, wl, cores)
            out["cpu_baseline"] = {"value": v, "unit": "butterflies/s", "cores": cores, "kind": "oracle",
                                   "sample": f"{cores} of the {wl['batch']} transforms (half forward, half "
                                             f"inverse), one per host thread, {dt:.1f} s wall"}
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Throughput of the LOFAR station-to-beam path on GB300: station-samples/s.

A step is one pass of the whole path (integer shift, 16-tap FIR + 256-point FFT, delay phase +
bandpass + corner turn, weights + tied-array beam former, Stokes + integration) over one block of
the workload through lbf_run_block.  Default workload: 48 stations (24 core in a 2 km disc, 24
remote to 80 km), 244 subbands of 195312.5 Hz, 196608-sample int16 blocks, 127 hex beams, Stokes I
integrated over 16 spectra, plain FP32 -- one 18.4 GB block per step (inputs larger than L2).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host cores
instead (bounded sample of the same workload).
"""

from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1105_0661_gb300 import dist  # noqa: E402
from synth import generate as G  # noqa: E402



def workload(name: str, subbands: int = 0, bits: int = 0):
    if name == "lofar":
        wl = G.workload_lofar_fp32(0)
    elif name == "lofar1024":
        wl = G.workload_lofar_tc(bits or 8, 0)
    elif name == "lofar8":
        # the same observation with 8 tied-array beams (the few-beam, bandwidth-bound beam former)
        wl = G.workload_lofar_fp32(0)
        wl.beam_dlm = G.hex_beam_grid(8, 0.05)
        wl.name = "lofar-48st-244sb-8beam-I16"
    elif name == "tiny":
        wl = G.workload_tiny(0)
    else:
        raise SystemExit(f"unknown workload {name}")
    if bits and bits != wl.sample_bits:
        wl.sample_bits = bits
        wl.sigma = 8.0 if bits == 8 else 32.0
        wl.name += f"-i{bits}"
    if 0 < subbands < wl.n_subbands:
        wl = wl.subset(list(range(subbands)))
    return wl


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = list(csv.reader(open(self.path)))
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline
def algorithmic_work(wl, dims):
    """Per-launch algorithmic bytes / flops of each kernel (the units the design notes state)."""
    S, F, T, B, M = wl.n_stations, wl.n_subbands, wl.block_samples, wl.n_beams, dims.n_spectra
    word = 8 if wl.sample_bits == 16 else 4
    ss = S * F * T                              # station-samples per block
    nS = dims.n_stokes
    out_bytes = B * max(nS, 1) * F * 256 * (M // wl.int_factor) * 4 if nS else B * F * T * 16
    return {
        "ppf_ct": ("hbm", ss * (word + 16)),    # read int samples, write 2 pols x cf32
        "ppf": ("hbm", ss * (word + 16)),
        "hist_update": ("hbm", 2 * S * F * dims.history_samples * word),
        "delay_ct": ("hbm", ss * 32),
        "bf_few": ("hbm", ss * 16 + out_bytes),  # read corner-turned cf32 once, write the output
        "bf_many": ("alu", 8.0 * B * ss * 2),   # 8 flop per complex MAC, B x S x 2 pols x T per subband
        "bf_many64": ("alu", 8.0 * B * ss * 2),
        "stokes": ("hbm", B * F * T * 16 + out_bytes),
        # FP16 forms: hi and lo half2 planes per pol; one complex product is the algorithmic work
        "ppf_ct16": ("hbm", ss * (word + 2 * 4 * 2)),
        "bf_tc": ("tensor", 8.0 * B * ss * 2),
        "ct_to_ct16": ("hbm", ss * (16 + 2 * 4 * 2)),
        "dedisperse": ("hbm", 2 * B * F * T * 16),   # read and write the voltages (2 pols x cf32)
    }


def traffic_from_profiles(kernel: str, workload_name: str):
    """DRAM bytes per launch recorded from an ncu capture of this workload, if the kernel source
    is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    src = {"bf_many": "beamform.cu", "bf_many64": "beamform.cu", "bf_few": "beamform.cu", "ppf_ct": "ppf.cu", "ppf": "ppf.cu",
           "ppf_ct16": "ppf.cu", "bf_tc": "bf_tc.cu", "hist_update": "ppf.cu", "delay_ct": "delay.cu",
           "dedisperse": "dedisperse.cu",
           "stokes": "stokes.cu", "superstation": "delay.cu"}.get(kernel)
    if src is None:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_1105_0661_gb300", "csrc", src), "rb").read()).hexdigest()[:16]
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 5 and cells[0] == kernel and cells[2] == h and workload_name.startswith(cells[3]):
            try:
                return float(cells[1])
            except ValueError:
                return None
    return None


def measure_alu_peak(stream, smi_index):
    """FP32 SIMT throughput of this GPU now (lbf_measure_fp32_peak) with the SM clock seen."""
    from paper_1105_0661_gb300 import lbf
    with ClockSampler(smi_index) as clk:
        r = lbf.measure_fp32_peak(5, stream)
        time.sleep(0.25)
    c = clk.summary()
    r["tflops"] = max(r["ffma_tflops"], r["ffma2_tflops"])
    r["clocks"] = f"{c['sm_mhz']:.0f} MHz median (max {c['sm_max_mhz']:.0f})" if c else "not sampled"
    return r


# ----------------------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    wl, f, blk = args
    from oracle import lbf_oracle
    t0 = time.perf_counter()
    out = lbf_oracle.observation_from_workload(wl.subset([f])).run_block(blk)
    return time.perf_counter() - t0, out


def run_oracle_sample(wl, blocks, subbands, workers):
    """Time the oracle on the given subbands (one process per subband, BLAS single-threaded).
    Returns (wall seconds, station-samples, per-subband outputs)."""
    env_keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, [(wl, f, b) for f, b in zip(subbands, blocks)])
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    ss = wl.n_stations * len(subbands) * wl.block_samples
    return wall, ss, [r[1] for r in res]


def host_block_slices(wl, seed, subbands):
    """Station data of the listed subbands, [S][1][T][2][2], drawn by the same seeded device
    generator the GPU arm uses (generated on the GPU when available, else as host noise)."""
    import numpy as np
    try:
        import torch
        if torch.cuda.is_available():
            from synth.device import make_block_device
            d = make_block_device(wl, seed, torch.device("cuda", torch.cuda.current_device()))
            out = [d[:, f:f + 1].cpu().numpy() for f in subbands]
            del d
            torch.cuda.empty_cache()
            return out
    except ImportError:
        pass
    return [G.make_block(wl.subset([f]), seed=seed, source="noise") for f in subbands]


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world = dist.init("gloo")
    if rank != 0:
        return 0
    wl = workload(args.workload, args.subbands, args.bits)
    nsub = min(args.cpu_subbands, wl.n_subbands)
    subbands = list(range(nsub))
    blocks = host_block_slices(wl, 0, subbands)
    for _ in range(args.warmup):
        run_oracle_sample(wl, blocks, subbands, nsub)
    times = []
    ss = 0
    for _ in range(args.steps):
        wall, ss, _ = run_oracle_sample(wl, blocks, subbands, nsub)
        times.append(wall)
    total = sum(times)
    value = ss * args.steps / total
    line = {
        "impl": "reference", "metric": "station-samples/s", "value": value, "unit": "station-samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(wl, args),
        "cpu_baseline": {"value": value, "unit": "station-samples/s", "cores": nsub, "kind": "oracle",
                         "sample": f"{nsub} of {wl.n_subbands} subbands x {wl.n_stations} stations x "
                                   f"{wl.block_samples} samples per step, whole path, FP64 numpy"},
        "e2e": {"value": value, "unit": "station-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(wl, args):
    return {"workload": wl.name, "stations": wl.n_stations, "subbands": wl.n_subbands,
            "block_samples": wl.block_samples, "channels": wl.n_channels, "taps": wl.n_taps,
            "beams": wl.n_beams, "output": wl.output, "int_factor": wl.int_factor,
            "sample_bits": wl.sample_bits, "precision": args.precision,
            "l2": "inputs larger than L2 (one block is %.1f GB)" % (wl.station_samples() * (8 if wl.sample_bits == 16 else 4) / 1e9),
            "parallelism": "independent observation per GPU (no collective)"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.build_lib import build
    from synth.device import make_block_device

    rank, local, world = dist.env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init("nccl" if world > 1 else "gloo")
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1105_0661_gb300", "_lib", "liblbf.so")):
        build()
    dist.barrier(dev)
    wl = workload(args.workload, args.subbands, args.bits)
    pk, pk_kind = peaks()
    args.cpu_subbands = min(args.cpu_subbands, wl.n_subbands)

    # cpu baseline first (spawned workers, before the large device allocations)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        subbands = list(range(args.cpu_subbands))
        blocks = host_block_slices(wl, 0, subbands)
        wall, ss, ref_out = run_oracle_sample(wl, blocks, subbands, args.cpu_subbands)
        cpu = {"value": ss / wall, "unit": "station-samples/s", "cores": args.cpu_subbands, "kind": "oracle",
               "sample": f"{args.cpu_subbands} of {wl.n_subbands} subbands x {wl.n_stations} stations x "
                         f"{wl.block_samples} samples (one block), whole path, FP64 numpy, one process per subband"}
    else:
        ref_out = None

    plan = Plan.from_workload(wl, precision=args.precision)
    dims = plan.dims
    d_in = make_block_device(wl, seed=rank, device=dev)
    out_dtype = torch.float32 if dims.n_stokes else torch.complex64
    d_out = torch.empty(plan.shape("stokes") if dims.n_stokes else plan.shape("vol"), dtype=out_dtype, device=dev)
    stream = torch.cuda.Stream(device=dev)

    # parity of the timed configuration on the oracle's sample (first block of a fresh stream)
    parity = None
    if ref_out is not None:
        plan.reset_state(stream)
        plan.run_block(d_in, d_out, stream)
        stream.synchronize()
        errs = []
        for f, ref in zip(range(args.cpu_subbands), ref_out):
            got = d_out[:, :, f:f + 1].double().cpu().numpy()
            I = ref[:, 0]
            errs.append(float((abs(got[:, 0] - I) / I).max()))
        parity = {"max_rel_err_stokes_I": max(errs), "subbands": args.cpu_subbands}

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = vis[local].strip() if len(vis) > local and vis[local].strip() else str(local)
    # the FP32 SIMT peak of this GPU, measured now (the denominator of the FP32 kernels' roofline)
    alu_peak = measure_alu_peak(stream, smi_index)

    for _ in range(args.warmup):
        plan.run_block(d_in, d_out, stream)
    stream.synchronize()
    dist.barrier(dev)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(smi_index) as clk:
        plan.trace_begin(3 * args.steps + 8)
        torch.cuda.synchronize(dev)
        dist.barrier(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            plan.run_block(d_in, d_out, stream)
        ev1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        dist.barrier(dev)
        trace = plan.trace_end()
    clocks = clk.summary()
    ms_local = ev0.elapsed_time(ev1)
    ms = dist.reduce_scalar(ms_local, "max", dev)
    ss_step = wl.station_samples()
    value = world * ss_step * args.steps / (ms / 1e3)

    # end to end through the multi-block host-buffer C-ABI call (pinned host memory; every block's
    # upload and download inside the timed region, uploads alternating between two device buffers)
    e2e = None
    if not args.no_e2e:
        h_in = torch.empty(d_in.shape, dtype=d_in.dtype, pin_memory=True)
        h_in.copy_(d_in)
        h_out = torch.empty(d_out.shape, dtype=d_out.dtype, pin_memory=True)
        d_stage = [torch.empty_like(d_in), torch.empty_like(d_in)]
        plan.run_blocks_host([h_in] * 2, [h_out] * 2, d_stage[0], d_stage[1], d_out, stream)
        stream.synchronize()

        # the pinned-copy rates of these buffers just before and just after the timed region (the
        # host link is shared with other jobs on the machine and varies between and within runs):
        # the end-to-end figure is read against them
        def copy_rates():
            r = {}
            for name, (dst, src) in {"h2d": (d_stage[0], h_in), "d2h": (h_out, d_out)}.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                dst.copy_(src, non_blocking=True)
                torch.cuda.synchronize()
                r[name] = src.numel() * src.element_size() / (time.perf_counter() - t0) / 1e9
            return r
        copy_before = copy_rates()
        dist.barrier(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # a stream of blocks: one upload fills the pipeline, so it is timed over at least 30 blocks
        k2 = max(args.steps, 30) if args.e2e_steps <= 0 else max(1, args.e2e_steps)
        e0.record(stream)
        plan.run_blocks_host([h_in] * k2, [h_out] * k2, d_stage[0], d_stage[1], d_out, stream)
        e1.record(stream)
        stream.synchronize()
        ems = dist.reduce_scalar(e0.elapsed_time(e1), "max", dev)
        copy_after = copy_rates()
        e2e = {"value": world * ss_step * k2 / (ems / 1e3), "unit": "station-samples/s",
               "h2d_bytes_per_step": dims.in_bytes, "d2h_bytes_per_step": dims.out_bytes,
               "steps": k2, "ms_per_step": ems / k2, "call": "lbf_run_blocks_host",
               "host_copy_gbs": {"before": copy_before, "after": copy_after}}
        del h_in, h_out, d_stage

    # roofline of the dominant kernel from the live trace
    work = algorithmic_work(wl, dims)
    kernels = {}
    total_ms = sum(v[1] for k, v in trace.items() if not k.startswith("_"))
    for k, v in trace.items():
        if k.startswith("_"):
            continue
        n, tms = v
        avg_s = tms / n / 1e3
        bound, amount = work[k]
        kernels[k] = {"launches": n, "avg_ms": tms / n, "share": tms / total_ms, "bound": bound}
        if bound in ("alu", "tensor"):
            kernels[k]["achieved_tflops"] = amount / avg_s / 1e12
        else:
            kernels[k]["achieved_gbs"] = amount / avg_s / 1e9
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    bound, amount = work[dom]
    avg_s = kernels[dom]["avg_ms"] / 1e3
    if bound == "tensor":
        # FP16 dense with FP32 accumulation: same nominal rate as BF16 (ratio 1), so the measured
        # sustained BF16 figure is the peak of a kernel timed inside a long step
        peak_tf = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        achieved = amount / avg_s / 1e12
        roof = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": traffic_from_profiles(dom, wl.name),
                "executed_tflops": achieved * 3,
                "peak_source": f"{pk_kind} bf16_tflops_sustained (fp16 dense nominal ratio 1.0); achieved counts "
                               f"one complex product, the hi+lo form executes three (Whi.Yhi + Whi.Ylo + Wlo.Yhi)"}
    elif bound == "alu":
        peak_tf = alu_peak["tflops"]
        achieved = amount / avg_s / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": traffic_from_profiles(dom, wl.name),
                "peak_source": "measured in this run: lbf_measure_fp32_peak, the faster of scalar FFMA "
                               f"({alu_peak['ffma_tflops']:.1f}) and packed FP32x2 ({alu_peak['ffma2_tflops']:.1f}) "
                               f"FMA chains on all {alu_peak['sms']} SMs, SM clock {alu_peak['clocks']}"}
    else:
        peak = pk["hbm_gbs"]
        achieved = amount / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(dom, wl.name),
                "peak_source": f"{pk_kind} hbm_gbs"}

    launches = sum(v[0] for k, v in trace.items() if not k.startswith("_")) + trace.get("_dropped", 0)
    bf_flop = 8.0 * wl.n_beams * ss_step * 2

    # the same block through the other precision form (the metric compares FP16-TC with FP32)
    compare = None
    if not args.no_compare and dims.n_stokes and wl.n_stations <= 64:
        other = "fp16tc" if args.precision == "fp32" else "fp32"
        plan.close()
        plan = Plan.from_workload(wl, precision=other)
        for _ in range(args.warmup):
            plan.run_block(d_in, d_out, stream)
        stream.synchronize()
        dist.barrier(dev)
        plan.trace_begin(3 * args.steps + 8)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            plan.run_block(d_in, d_out, stream)
        c1.record(stream)
        stream.synchronize()
        ctrace = plan.trace_end()
        cms = dist.reduce_scalar(c0.elapsed_time(c1), "max", dev)
        bf_ms = sum(v[1] for k, v in ctrace.items() if k.startswith("bf_"))
        compare = {"precision": other, "value": world * ss_step * args.steps / (cms / 1e3),
                   "ms_per_step": cms / args.steps,
                   "kernels_ms": {k: v[1] / v[0] for k, v in ctrace.items() if not k.startswith("_") and v[0]},
                   "beamform_tflops": bf_flop * args.steps / (bf_ms / 1e3) / 1e12,
                   "speedup_of_fp16tc": (ms / cms) if other == "fp16tc" else (cms / ms)}
        launches_other = sum(v[0] for k, v in ctrace.items() if not k.startswith("_"))
        compare["gpu_launches"] = launches_other
    line = {
        "metric": "station-samples/s", "value": value, "unit": "station-samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f16", "data": "synthetic",
        "config": config_dict(wl, args), "e2e": e2e, "gpu_launches": launches, "roofline": roof,
        "cpu_baseline": cpu, "clocks": clocks, "kernels": kernels, "fp32_peak": alu_peak,
        "beamform_tflops": bf_flop * args.steps / (sum(v[1] for k, v in trace.items() if k.startswith("bf_")) / 1e3) / 1e12,
        "dtype_detail": {"fp16tc": "fp16 tensor-core operands (three products), fp32 accumulation",
                         "fp16tc2": "fp16 tensor-core operands (two products), fp32 accumulation"}.get(args.precision, "fp32"),
        "parity": parity, "precision_compare": compare,
        "paper_context": "Blue Gene/P rack: up to 198 Gb/s = 3.1e9 station-samples/s (64 stations x 248 subbands)",
    }
    plan.close()
    del d_in, d_out
    torch.cuda.empty_cache()
    # the metric's other two parts on the same GPU, rank 0 at N = 1: the 1024-beam precision form
    # (FP16 tensor cores vs plain FP32) and the serving loop's p99 block latency
    if rank == 0 and world == 1 and not args.no_extras:
        line["precision_form_1024beam"] = precision_form_1024(args, dev, stream, pk, smi_index)
        line["serving"] = serve_measure(dev, args.serve_obs, args.serve_line_blocks, args.budget_gb,
                                        args.serve_chunks, smi_index)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier(dev)
    dist.finalize()
    return 0


# ----------------------------------------------------------------------------- serving
def serving_observations(n: int, seed: int = 5):
    """The streaming workload: n observations with stations 24-64, subbands 61-244, beams 7-1024,
    Stokes I or IQUV (integration 16), 196608-sample int16 blocks, drawn from a seeded rng.  Every
    plan asks for the tensor-core precision; the library keeps the tensor cores for more than 8
    beams and gives fewer beams the bandwidth-bound FP32 few-beam kernel."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S = int(rng.integers(24, 65))
        F = int(rng.integers(61, 245))
        B = int(np.exp(rng.uniform(np.log(7), np.log(1024))))
        kind = "IQUV" if rng.random() < 0.5 else "I"
        xyz = G.lofar_positions(rng, S // 2, S - S // 2)
        wl = G.Workload(f"serve{i}-{S}st-{F}sb-{B}beam-{kind}16", xyz, G.subband_centres(F, 110e6),
                        G.hex_beam_grid(B, 0.05), (0.3, 0.4), 196608, 16, kind, source="noise")
        out.append((wl, "fp16tc" if S <= 64 else "fp32"))
    return out


def serve_measure(dev, n_obs: int, n_blocks: int, budget_gb: float, n_chunks: int, smi_index: str = "0") -> dict:
    """The streaming server on the serving workload: n_obs observations, n_blocks blocks each at
    the real-time period with late-arrival jitter, each observation served in n_chunks subband
    chunks.  Returns latencies, sustained throughput, the host link's copy rates, kernel time per
    period and the clocks seen."""
    import numpy as np
    import torch

    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.serve import Server, latency_summary, poisson_schedule, subband_ranges
    from synth.device import make_block_device

    period = 196608 / G.SUBBAND_RATE_HZ
    specs = serving_observations(n_obs)
    srv = Server(dev, int(budget_gb * 1e9))
    chunk_plans = []
    for wl, prec in specs:
        chunk_plans.append([(Plan.from_workload(wl.subset(list(range(f, f + n))), precision=prec,
                                                external_workspace=True), f)
                            for f, n in subband_ranges(wl.n_subbands, n_chunks)])
    in_b = [sum(p.dims.in_bytes for p, _ in cp) for cp in chunk_plans]
    out_b = [sum(p.dims.out_bytes for p, _ in cp) for cp in chunk_plans]
    # one pinned host input/output area serves every observation (block contents do not change
    # the work; they are synthetic noise of the right shape, copied in each step)
    h_in = torch.empty(max(in_b), dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(max(out_b), dtype=torch.uint8, pin_memory=True)
    big = max(specs, key=lambda x: x[0].station_samples())[0]
    blk = make_block_device(big, 0, dev)
    h_in[:blk.numel() * blk.element_size()].copy_(blk.view(torch.uint8).reshape(-1))
    del blk
    torch.cuda.empty_cache()

    # the host-copy rates of this process's pinned buffers (the server's copies are most of its
    # per-block time), before and after the schedule
    def copy_rates():
        r = {}
        nb = min(max(in_b), 4 << 30)
        d_probe = torch.empty(nb, dtype=torch.uint8, device=dev)
        for name, (dst, src) in {"h2d": (d_probe, h_in[:nb]), "d2h": (h_in[:nb], d_probe)}.items():
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            r[name] = nb / (time.perf_counter() - t0) / 1e9
        del d_probe
        torch.cuda.empty_cache()
        return r
    copy_before = copy_rates()
    for oid, cp in enumerate(chunk_plans):
        srv.add(oid, cp, specs[oid][0].n_subbands, h_in, h_out)
    # warm-up: one block per observation, outside the measured schedule
    srv.run([(0.0, oid, -1) for oid in range(len(specs))])
    for o in srv.obs.values():
        o.results.clear()
    rng = np.random.default_rng(11)
    sched = poisson_schedule(len(specs), n_blocks, period, rng)
    # kernel times of every chunk plan and the clocks while the schedule runs, so that a slow run
    # can be told apart from a slow host link
    plans = [p for cp in chunk_plans for p, _ in cp]
    for p in plans:
        p.trace_begin(8 * n_blocks + 8)
    with ClockSampler(smi_index) as clk:
        res, wall = srv.run(sched)
    kernel_ms, launches = {}, 0
    for p in plans:
        for k, v in p.trace_end().items():
            if k.startswith("_") or not v[0]:
                continue
            kernel_ms[k] = kernel_ms.get(k, 0.0) + v[1]
            launches += v[0]
    copy_after = copy_rates()
    summ = latency_summary(res, period)
    ss = sum(specs[r.obs][0].station_samples() for r in res)
    first = min(r.arrival for r in res)
    last = max(r.done for r in res)
    out = {
        "latency": summ,
        # served station-samples over the span from the first arrival to the last completion
        # (with few blocks per observation the span includes the ramp-up of the staggered
        # observations and the drain of the last blocks, so it reads below the arrival rate)
        "sustained_station_samples_per_s": ss / (last - first),
        # fraction of that span with a block waiting or in flight: below 1 with no late block,
        # the server keeps up with the arrivals and has capacity left
        "busy_fraction": srv.busy_s / (last - first),
        "capacity_station_samples_per_s": ss / srv.busy_s if srv.busy_s > 0 else None,
        "realtime_station_samples_per_s": sum(wl.station_samples() for wl, _ in specs) / period,
        "host_copy_gbs": {"before": copy_before, "after": copy_after},
        "kernel_s_per_period": sum(kernel_ms.values()) / 1e3 / (wall / period), "kernels_ms_total": kernel_ms,
        "clocks": clk.summary(), "period_s": period, "hbm_budget_gb": budget_gb, "chunks_per_observation": n_chunks,
        "observations": [wl.name + f" ({'tensor cores' if p.dims.bf_kernel == 3 else 'fp32'})"
                         for (wl, _), p in zip(specs, [cp[0][0] for cp in chunk_plans])],
        "mean_h2d_bytes_per_block": int(np.mean(in_b)), "mean_d2h_bytes_per_block": int(np.mean(out_b)),
        "gpu_launches": launches,
    }
    for p in plans:
        p.close()
    del srv, h_in, h_out
    torch.cuda.empty_cache()
    return out


def run_serve(args):
    import torch

    from paper_1105_0661_gb300.build_lib import build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = serve_measure(dev, args.serve_obs, args.serve_blocks, args.budget_gb, args.serve_chunks)
    summ = r["latency"]
    line = {
        "metric": "p99 block latency", "value": summ["p99_s"], "unit": "s", "n_gpus": 1,
        "steps": summ["blocks"], "warmup": args.serve_obs, "ms_per_step": 1e3 * summ["p50_s"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f16",
        "data": "synthetic",
        "config": {"workload": f"serving: {args.serve_obs} observations, 196608-sample int16 blocks at the "
                               f"real-time period with late-arrival jitter (exponential, mean period/4)",
                   "observations": r["observations"], "hbm_budget_gb": args.budget_gb, "period_s": r["period_s"],
                   "chunks_per_observation": args.serve_chunks},
        **{k: v for k, v in r.items() if k not in ("observations",)},
        "e2e": {"value": summ["p99_s"], "unit": "s", "h2d_bytes_per_step": r["mean_h2d_bytes_per_block"],
                "d2h_bytes_per_step": r["mean_d2h_bytes_per_block"]},
    }
    print(json.dumps(line), flush=True)
    return 0


def precision_form_1024(args, dev, stream, pk, smi_index):
    """The precision form of the observation (1024 beams on a hexagonal grid, full Stokes IQUV
    integrated over 16): FP16 tensor cores with int8 samples and with int16 samples, in the
    three-product form and the two-product form (FP16 weights), and the plain FP32 path on the same
    int8 block."""
    import torch

    from paper_1105_0661_gb300 import Plan
    from synth.device import make_block_device

    res = {}
    peak_tf = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    with ClockSampler(smi_index) as clk:
        for bits in (8, 16):
            wl = G.workload_lofar_tc(bits, 0)
            d_in = make_block_device(wl, seed=0, device=dev)
            ss = wl.station_samples()
            flop = 8.0 * wl.n_beams * ss * 2               # one complex product per MAC
            forms = ("fp16tc", "fp16tc2", "fp32") if bits == 8 else ("fp16tc", "fp16tc2")
            for prec in forms:
                plan = Plan.from_workload(wl, precision=prec)
                d_out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
                steps = args.steps if prec != "fp32" else 2
                for _ in range(3):
                    plan.run_block(d_in, d_out, stream)
                stream.synchronize()
                plan.trace_begin(4 * steps + 8)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    plan.run_block(d_in, d_out, stream)
                e1.record(stream)
                stream.synchronize()
                tr = plan.trace_end()
                ms = e0.elapsed_time(e1) / steps
                r = {"ms_per_step": ms, "value": ss / (ms / 1e3), "steps": steps, "warmup": 3,
                     "kernels_ms": {k: v[1] / v[0] for k, v in tr.items() if not k.startswith("_") and v[0]}}
                bf = "bf_tc" if prec != "fp32" else ("bf_many" if "bf_many" in r["kernels_ms"] else "bf_few")
                bf_ms = r["kernels_ms"].get(bf)
                if bf_ms:
                    r["beamform_tflops"] = flop / (bf_ms / 1e3) / 1e12
                    if prec != "fp32":   # executed: three (fp16tc) or two (fp16tc2) FP16 products
                        r["bf_tc_frac_algorithmic"] = r["beamform_tflops"] / peak_tf
                        r["bf_tc_frac_executed"] = (3 if prec == "fp16tc" else 2) * r["beamform_tflops"] / peak_tf
                        r["peak_tflops"] = peak_tf
                res[f"{prec}_i{bits}"] = r
                plan.close()
                del d_out
                torch.cuda.empty_cache()
            del d_in
            torch.cuda.empty_cache()
    res["fp16tc_speedup_over_fp32_i8"] = res["fp32_i8"]["ms_per_step"] / res["fp16tc_i8"]["ms_per_step"]
    res["fp16tc2_speedup_over_fp32_i8"] = res["fp32_i8"]["ms_per_step"] / res["fp16tc2_i8"]["ms_per_step"]
    res["workload"] = "48 st x 244 sb x 196608 samples, 1024 hex beams, Stokes IQUV over 16 spectra"
    res["clocks"] = clk.summary()
    return res


# ----------------------------------------------------------------------------- batching
def batch_observations(n: int = 16):
    """The batched workload (16 uneven sub-observations, 65536-sample blocks; synth.generate)."""
    return G.batch_workloads(n, 65536)


# ----------------------------------------------------------------------------- pulsar pipeline
def run_dedisperse(args):
    """Beam voltages at full bandwidth (complex-voltage output), channel-level dedispersion
    (Section 4.4) in place, then Stokes I: the LOFAR observation with 127 beams."""
    import torch

    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.build_lib import build
    from synth.device import make_block_device

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pk, pk_kind = peaks()
    wl = workload(args.workload, args.subbands, args.bits)
    wl_v = G.Workload(**{**wl.__dict__, "output": "V", "name": wl.name + "-voltages"})
    pv = Plan.from_workload(wl_v, precision=args.precision)
    ps = Plan.from_workload(wl)
    d_in = make_block_device(wl, seed=0, device=dev)
    vol = torch.empty(pv.shape("vol"), dtype=torch.complex64, device=dev)
    out = torch.empty(ps.shape("stokes"), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    K, dm = args.dd_fft, args.dm

    def step():
        pv.run_block(d_in, vol, stream)
        pv.dedisperse(dm, K, vol, vol, stream)
        ps.stokes(vol, out, stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler("0") as clk:
        pv.trace_begin(4 * args.steps + 8)
        ps.trace_begin(2 * args.steps + 8)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        stream.synchronize()
        trace = pv.trace_end()
        trace_s = ps.trace_end()
    ms = ev0.elapsed_time(ev1) / args.steps
    ss = wl.station_samples()
    dims = pv.dims
    work = algorithmic_work(wl_v, dims)
    work["stokes"] = ("hbm", dims.vol_bytes + ps.dims.stokes_bytes)
    kernels = {}
    for tr in (trace, trace_s):
        for k, v in tr.items():
            if k.startswith("_") or not v[0]:
                continue
            n, tms = v
            bound, amount = work[k]
            avg_s = tms / n / 1e3
            kernels[k] = {"launches": n, "avg_ms": tms / n, "bound": bound}
            kernels[k]["achieved_tflops" if bound in ("alu", "tensor") else "achieved_gbs"] = \
                amount / avg_s / (1e12 if bound in ("alu", "tensor") else 1e9)
    dd = kernels["dedisperse"]
    line = {
        "metric": "station-samples/s", "value": ss / (ms / 1e3), "unit": "station-samples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f16+f32",
        "data": "synthetic",
        "config": {"workload": f"pulsar pipeline: {wl.name}, voltages ({args.precision}) -> channel-level dedispersion "
                               f"({K}-point FFT, DM {dm}) -> Stokes {wl.output} over {wl.int_factor}",
                   "voltage_bytes": dims.vol_bytes, "l2": "inputs larger than L2"},
        "gpu_launches": sum(v["launches"] for v in kernels.values()),
        "roofline": {"bound": "hbm", "kernel": "dedisperse", "achieved": dd["achieved_gbs"], "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": dd["achieved_gbs"] / pk["hbm_gbs"],
                     "traffic": traffic_from_profiles("dedisperse", wl.name),
                     "peak_source": f"{pk_kind} hbm_gbs"},
        "kernels": kernels, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    pv.close()
    ps.close()
    return 0


# ----------------------------------------------------------------------------- Section 8(f) rows
def run_superstation(args):
    """Superstation beam former (Section 4.2) on the LOFAR observation's corner-turned block:
    48 stations summed in 24 pairs; HBM-bound (read every station, write every group)."""
    import numpy as np
    import torch

    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.build_lib import build

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pk, pk_kind = peaks()
    wl = workload(args.workload, args.subbands, args.bits)
    plan = Plan.from_workload(wl)
    S = wl.n_stations
    groups = np.arange(S) // 2
    G_n = int(groups.max()) + 1
    gen = torch.Generator(device=dev).manual_seed(0)
    ct = torch.randn(plan.shape("ct"), dtype=torch.complex64, device=dev, generator=gen)
    F, N, _, P, M = plan.shape("ct")
    ss = torch.empty((F, N, G_n, P, M), dtype=torch.complex64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        plan.superstation(groups, ct, ss, stream)
    stream.synchronize()
    with ClockSampler("0") as clk:
        plan.trace_begin(args.steps + 8)
        for _ in range(args.steps):
            plan.superstation(groups, ct, ss, stream)
        stream.synchronize()
        tr = plan.trace_end()
    n, tms = tr["superstation"]
    avg_s = tms / n / 1e3
    nbytes = ct.numel() * 8 + ss.numel() * 8
    gbs = nbytes / avg_s / 1e9
    line = {
        "metric": "station-samples/s", "value": wl.station_samples() / avg_s, "unit": "station-samples/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tms / n, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"superstations: {wl.name} corner-turned block, {S} stations in {G_n} groups of 2",
                   "l2": "inputs larger than L2 (%.1f GB read per step)" % (ct.numel() * 8 / 1e9)},
        "gpu_launches": n,
        "roofline": {"bound": "hbm", "kernel": "superstation", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / pk["hbm_gbs"], "traffic": traffic_from_profiles("superstation", wl.name),
                     "peak_source": f"{pk_kind} hbm_gbs"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_incoherent(args):
    """Cost of the incoherent beam (Section 3) on the LOFAR block, fused into the FP32 many-beam
    kernel and as a separate kernel on the tensor-core path: steps with and without it."""
    import torch

    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.build_lib import build
    from synth.device import make_block_device

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = workload(args.workload, args.subbands, args.bits)
    d_in = make_block_device(wl, seed=0, device=dev)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for prec in ("fp32", "fp16tc"):
        for inc in (False, True):
            plan = Plan.from_workload(wl, precision=prec, incoherent_beam=inc)
            out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
            for _ in range(args.warmup):
                plan.run_block(d_in, out, stream)
            stream.synchronize()
            plan.trace_begin(4 * args.steps + 8)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                plan.run_block(d_in, out, stream)
            e1.record(stream)
            stream.synchronize()
            tr = plan.trace_end()
            res[f"{prec}{'_incoherent' if inc else ''}"] = {
                "ms_per_step": e0.elapsed_time(e1) / args.steps,
                "kernels_ms": {k: v[1] / v[0] for k, v in tr.items() if not k.startswith("_") and v[0]}}
            plan.close()
            del out
    line = {
        "metric": "station-samples/s", "value": wl.station_samples() / (res["fp32_incoherent"]["ms_per_step"] / 1e3),
        "unit": "station-samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["fp32_incoherent"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{wl.name} with the incoherent beam appended (Stokes {wl.output})"},
        "runs": res,
        "overhead_fp32": res["fp32_incoherent"]["ms_per_step"] / res["fp32"]["ms_per_step"] - 1.0,
        "overhead_fp16tc": res["fp16tc_incoherent"]["ms_per_step"] / res["fp16tc"]["ms_per_step"] - 1.0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    import torch

    from paper_1105_0661_gb300 import Batch, Plan
    from paper_1105_0661_gb300.build_lib import build
    from synth.device import make_block_device

    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wls = G.small_batch_workloads() if args.batch_small else batch_observations(16)
    # --precision fp16tc: observations with >= 64 beams and <= 64 stations on the tensor cores (as
    # the serving path chooses), the rest FP32; the separate launches use the same plans
    prec = ["fp16tc" if (args.precision == "fp16tc" and wl.n_beams >= 64 and wl.n_stations <= 64) else "fp32"
            for wl in wls]
    plans = [Plan.from_workload(wl, precision=pr) for wl, pr in zip(wls, prec)]
    d_in = [make_block_device(wl, seed=i + 1, device=dev) for i, wl in enumerate(wls)]
    d_out = [torch.empty(p.dims.out_bytes // 4, dtype=torch.float32, device=dev) for p in plans]
    stream = torch.cuda.Stream(device=dev)
    ss = sum(wl.station_samples() for wl in wls)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    def separate():
        for p, a, b in zip(plans, d_in, d_out):
            p.run_block(a, b, stream)

    ms_sep = timed(separate, args.steps)
    batch = Batch(plans)
    tuning = batch.tune(d_in, d_out, reps=2, stream=stream)
    batch.capture(d_in, d_out, stream=stream)
    ms_graph = timed(lambda: batch.launch(stream), args.steps)
    line = {
        "metric": "station-samples/s", "value": ss / (ms_graph / 1e3), "unit": "station-samples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f32+f16",
        "data": "synthetic",
        "config": {"workload": ("batched: 64 small observations (stations 8-16, subbands 2-8, beams 1-8, int16, "
                                "seed 5), 16384-sample blocks, Stokes I over 4") if args.batch_small else
                               ("batched: 16 sub-observations (stations 12-64, subbands 8-244, beams 1-512, "
                                "int8/int16, seeds 1-16), 65536-sample blocks, Stokes I over 4"),
                   "observations": [f"{wl.name} ({pr})" for wl, pr in zip(wls, prec)],
                   "l2": "inputs larger than L2 (%.1f GB per step)" % (sum(p.dims.in_bytes for p in plans) / 1e9)},
        "separate_launches": {"value": ss / (ms_sep / 1e3), "ms_per_step": ms_sep, "gpu_launches": 3 * len(plans)},
        "precision": args.precision,
        "speedup_vs_separate": ms_sep / ms_graph, "tuning": tuning,
        "gpu_launches": batch.launches(),
    }
    print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lofar", choices=["lofar", "lofar1024", "lofar8", "tiny"])
    ap.add_argument("--bits", type=int, default=0, choices=[0, 8, 16], help="sample width override")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16tc", "fp16tc2"])
    ap.add_argument("--subbands", type=int, default=0,
                    help="use only the first N subbands (small profiling cases; 0 = all)")
    ap.add_argument("--cpu-subbands", type=int, default=0,
                    help="subbands in the oracle sample, one process each (default: one per host core, <= 16)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end blocks in the streaming host call (0: max(K, 30))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other precision form on the same block")
    ap.add_argument("--serve", action="store_true", help="streaming serving run (p50/p99 block latency)")
    ap.add_argument("--batch", action="store_true", help="16 uneven sub-observations, grouped graph vs separate")
    ap.add_argument("--batch-small", action="store_true",
                    help="with --batch: 64 small observations instead (where grouped launches pay)")
    ap.add_argument("--dedisperse", action="store_true",
                    help="voltages -> channel-level dedispersion -> Stokes (pulsar pipeline)")
    ap.add_argument("--dd-fft", type=int, default=256, help="dedispersion FFT length (spectra)")
    ap.add_argument("--superstation", action="store_true", help="superstation beam former on the corner-turned block")
    ap.add_argument("--incoherent", action="store_true", help="cost of the incoherent beam on both precision paths")
    ap.add_argument("--dm", type=float, default=13.8, help="dispersion measure, pc cm^-3")
    ap.add_argument("--serve-obs", type=int, default=8)
    ap.add_argument("--serve-blocks", type=int, default=16)
    ap.add_argument("--serve-line-blocks", type=int, default=12,
                    help="blocks per observation of the serving run inside the default bench line")
    ap.add_argument("--serve-chunks", type=int, default=4, help="subband chunks per served observation")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the 1024-beam precision form and the serving run")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.cpu_subbands <= 0:   # one oracle process per subband, one per host core
        args.cpu_subbands = min(16, os.cpu_count() or 4)
    if args.warmup < 3:
        print("bench: warm-up must be >= 3 steps", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.batch:
        return run_batch(args)
    if args.dedisperse:
        return run_dedisperse(args)
    if args.superstation:
        return run_superstation(args)
    if args.incoherent:
        return run_incoherent(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

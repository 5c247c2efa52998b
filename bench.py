#!/usr/bin/env python3
"""Benchmark of the CKKS hot path on GB300.

Headline metric: negacyclic NTT limb-transforms per second at N = 2^15 on the
paper's NTT workload (1024 instances x 8 RNS limbs; 60- and 50-bit primes),
batched (one launch per direction for all 8192 limbs). A step is one forward
and one inverse transform of the whole batch, in place, inputs resident in
HBM (2 GiB per direction, far larger than the 129 MB L2, so no flush is
needed). The same run also measures, as sub-results:
  * the plain form (one launch per polynomial) and the CUDA-graph form;
  * the naive radix-2 baseline of the paper (one launch per stage);
  * mul-relin-rescale (MulLinRS) per second on the CKKS workload (N = 16384,
    one 60-bit + six 50-bit data primes, 60-bit special prime, 64 ciphertext
    pairs), batched versus one call per pair;
  * the end-to-end NTT rate through host buffers: every step one
    he_ntt_host call copies the batch from pinned host memory, runs forward
    and inverse and copies it back, pipelined in chunks over four streams
    (and, for comparison, the same with one whole-batch copy each way);
  * the register-resident butterfly probe (integer roof) and the roofline of
    the forward transform kernel;
  * the CPU oracle on a bounded sample (cpu_baseline).

`--impl reference` times the CPU oracle alone on the same metric.
Under torchrun each rank runs the full workload on its own GPU (independent
replicas; the transform needs no communication) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
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

NTT_LOG_N = 15
NTT_LIMBS = 8
NTT_INSTANCES = 1024
MRR_N = 16384
MRR_BITS = [60] + [50] * 6
MRR_COUNT = 64
METRIC = "NTT limbs/s at N=2^15 + HE mul-relin-rescale/s, batched vs plain; p99 latency"
# DRAM bytes (read + write) of one launch of the 1024 x 8 x 2^15 batch, per
# direction and transform shape (log_block, log_thread_words, persistent):
# an ncu capture of the same kernel on 256 instances scaled by 4 (traffic
# grows in proportion to the limbs). Entries are removed when the kernel
# changes after their capture, so that no stale figure is reported.
TRAFFIC = {
    ("forward", (12, 4, 0, 0)): 4 * (542030000 + 475360000),
    ("inverse", (12, 4, 0, 0)): 4 * (542990000 + 476230000),
}
# The production forward butterfly keeps the IMAD (fmaheavy) pipe busy for
# 0.2536 cycles per butterfly per SM: ncu on the register-resident probe
# (1216 x 256 threads x 16 x 1024 butterflies) counts that pipe 94.2 % active
# over 9.034 M cycles, i.e. 8.51 M busy cycles for 33.55 M butterflies per SM.
# It is the binding unit (issue slots are 61 % used), so the integer peak is
# SMs x clock / FMAHEAVY_CYCLES_PER_BFLY butterflies per second.
FMAHEAVY_CYCLES_PER_BFLY = 0.2536
UNIT = "limb-NTT/s"
CPU_RUNS = 5                          # the CPU baseline is the median of this many runs
REF_INSTANCES = NTT_INSTANCES // 8    # reference arm: 1/8 of the batch per step
TUNE_REPS = 10                        # autotuner: median of this many timed runs per candidate


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    ap.add_argument("--profile-case", choices=["ntt", "mrr", "mrr_multi", "probe", "encode", "product"],
                    help="run one small case of a kernel family and exit (for profilers)")
    ap.add_argument("--instances", type=int, default=64,
                    help="NTT instances of --profile-case ntt, ciphertext pairs of --profile-case mrr")
    ap.add_argument("--shape", default="",
                    help="log_block,log_thread_words[,persistent] for --profile-case ntt (or fwd/inv)")
    ap.add_argument("--skip", default="",
                    help="comma list of sub-benchmarks to skip: small,degrees,uneven,matrix,routines,encode,serving")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--no-tune-cache", action="store_true", help="always re-run the autotuner")
    ap.add_argument("--ref-instances", type=int, default=REF_INSTANCES,
                    help="instances per step of the reference arm (default: 1/8 of the batch)")
    a = ap.parse_args()
    a.skip = set(x for x in a.skip.split(",") if x)
    return a


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _ntt_moduli(cpu_oracle: bool = False):
    """Four 60-bit then four 50-bit primes = 1 mod 2N (the CPU legs take the
    oracle's own prime search, the GPU leg the library's; both give the same
    primes)."""
    two_n = 2 << NTT_LOG_N
    if cpu_oracle:
        import oracle
        return oracle.find_primes(60, two_n, NTT_LIMBS // 2) + oracle.find_primes(50, two_n, NTT_LIMBS // 2)
    from paper_2109_14704_gb300 import he
    return he.primes_generate(60, two_n, NTT_LIMBS // 2) + he.primes_generate(50, two_n, NTT_LIMBS // 2)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed regions run."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "util": float(parts[4]),
                             "hw": parts[6], "hw_th": parts[7], "sw_th": parts[8], "pcap": parts[9]})
            except ValueError:
                continue
        os.unlink(self.path)
        loaded = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in loaded:
            for key, name in (("hw", "hw_slowdown"), ("hw_th", "hw_thermal_slowdown"),
                              ("sw_th", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded) if loaded else None,
                "sm_max_mhz": max(r["max"] for r in loaded) if loaded else None,
                "reasons": sorted(reasons), "samples": len(loaded)}


# ---------------------------------------------------------- GPU timing

def _time_steps(fn, steps, warmup, stream, barrier):
    import torch
    for _ in range(warmup):
        fn()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return t0.elapsed_time(t1) / steps


def _distribution(ms_list) -> dict:
    """Median, p99, extremes and count of single-step times (ms)."""
    import numpy as np
    xs = sorted(ms_list)
    return {"median_ms": statistics.median(xs), "p99_ms": float(np.percentile(xs, 99)), "min_ms": xs[0],
            "max_ms": xs[-1], "reps": len(xs)}


def _step_times(fn, reps, stream) -> list:
    """Each call timed alone with CUDA events on the launching stream."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _collectives(world: int, device):
    """(barrier, max_over_ranks) over the initialised process group (any
    backend; `device` holds the reduction tensor), or no-ops for one rank.
    Replicas share nothing else: the timed step takes the slowest rank's
    time and the job value counts every rank's work."""
    if world <= 1:
        return (lambda: None), (lambda x: x)
    import torch
    import torch.distributed as dist

    def barrier():
        dist.barrier()

    def max_over_ranks(x):
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def job_value(world: int, units_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def mrr_work(n: int, N: int) -> dict:
    """Algorithmic work of one MulLinRS (tensor, relinearization with one
    special prime and n RNS digits, rescale) at n data limbs and degree N:
    n^2 + 5n + 2 transforms of (N/2) log2 N butterflies; N (2n^2 + 16n - 4)
    further modular products (tensor 4n, key products 2n(n+1), d P 2n,
    mod-down 2n + 2n centred reductions, rescale 2(n-1) + 2(n-1)); HBM bytes:
    the two input ciphertexts read and the output written once (the
    resident key is not counted)."""
    log_n = N.bit_length() - 1
    return {"bfly": (n * n + 5 * n + 2) * (N // 2) * log_n, "products": N * (2 * n * n + 16 * n - 4),
            "bytes": (4 * n + 2 * (n - 1)) * N * 8}


def roof_entry(work: dict, seconds: float, alu_peak: float, hbm_peak: float) -> dict:
    """Achieved rates of `work` (bfly, products, bytes per timed unit of
    `seconds`) against the derived integer peak (butterflies/s) and the
    measured HBM copy bandwidth (GB/s). A modular product outside the
    transforms is counted as one butterfly (one Shoup-sized multiply)."""
    e = {"tbfly_per_s": work["bfly"] / seconds / 1e12, "alu_frac_transforms": work["bfly"] / seconds / alu_peak,
         "gbs": work["bytes"] / seconds / 1e9, "hbm_frac": work["bytes"] / seconds / 1e9 / hbm_peak}
    if work.get("products"):
        e["alu_frac_with_products"] = (work["bfly"] + work["products"]) / seconds / alu_peak
    return e


def attach_rooflines(obj, alu_peak: float, hbm_peak: float):
    """Replace every "_work" entry ({"bfly", "products", "bytes", "seconds"})
    in a (nested) result by its "roofline" entry."""
    if isinstance(obj, dict):
        w = obj.pop("_work", None)
        if w is not None:
            obj["roofline"] = roof_entry(w, w["seconds"], alu_peak, hbm_peak)
        for v in obj.values():
            attach_rooflines(v, alu_peak, hbm_peak)
    elif isinstance(obj, list):
        for v in obj:
            attach_rooflines(v, alu_peak, hbm_peak)
    return obj


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import autotune, he
    from paper_2109_14704_gb300.synth import Rng

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    barrier, max_over_ranks = _collectives(world, dev)

    he.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    N = 1 << NTT_LOG_N
    qs = _ntt_moduli()
    tables = he.NttTables(N, qs)
    r = Rng(1000 + rank)
    host = np.stack([r.uniform_limbs(qs, N) for _ in range(NTT_INSTANCES)])
    pinned = torch.from_numpy(host.view(np.int64)).pin_memory()
    d = torch.empty(pinned.shape, dtype=torch.int64, device=dev)
    d.copy_(pinned)
    limbs_total = NTT_INSTANCES * NTT_LIMBS
    bytes_per_launch = 16 * N * limbs_total          # read + write every word once

    def step_batched():
        he.ntt_fwd(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        he.ntt_inv(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)

    # pick the transform shape for this batch (checked, timed, applied)
    tune = autotune.tune_uniform(N, NTT_LIMBS, NTT_INSTANCES, moduli=qs, reps=TUNE_REPS, warmup=3,
                                 cache_path=None if args.no_tune_cache else autotune.DEFAULT_CACHE)
    d.copy_(pinned)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    ms = _time_steps(step_batched, args.steps, args.warmup, stream, barrier)
    ms = max_over_ranks(ms)

    # per-kernel durations for the roofline (events on the launching stream),
    # and from them the distribution of single steps (median and p99 over at
    # least 20; inputs of 2 GiB, larger than L2)
    fwd_ms, inv_ms = [], []
    for _ in range(max(20, args.steps)):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        he.ntt_fwd(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        e[1].record(stream)
        he.ntt_inv(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwd_ms.append(e[0].elapsed_time(e[1]))
        inv_ms.append(e[1].elapsed_time(e[2]))
    fwd = statistics.mean(fwd_ms)
    inv = statistics.mean(inv_ms)
    step_dist = _distribution([a + b for a, b in zip(fwd_ms, inv_ms)])

    # CUDA-graph form of the batched step
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step_batched()
        with torch.cuda.graph(g, stream=side):
            he.ntt_fwd(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=side)
            he.ntt_inv(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    ms_graph = _time_steps(g.replay, args.steps, args.warmup, stream, barrier)

    # plain form: one launch per polynomial (8 limbs), as a per-polynomial API
    per_poly = [d[p] for p in range(NTT_INSTANCES)]

    def step_plain():
        for t in per_poly:
            he.ntt_fwd(t, N, NTT_LIMBS, 1, tables, stream=stream)
        for t in per_poly:
            he.ntt_inv(t, N, NTT_LIMBS, 1, tables, stream=stream)

    ms_plain = _time_steps(step_plain, max(2, args.steps // 5), 3, stream, barrier)

    # the paper's naive radix-2 baseline (one launch per stage)
    def step_naive():
        he.ntt_fwd_naive(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        he.ntt_inv_naive(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)

    ms_naive = _time_steps(step_naive, max(2, args.steps // 5), 3, stream, barrier)

    # MulLinRS on the CKKS evaluation workload
    data, P = he.chain_primes(MRR_N, MRR_BITS, 60)
    ctx = he.Context(MRR_N, data, P)
    L = len(data) - 1
    rm = Rng(2000 + rank)
    evk = np.stack([np.stack([rm.uniform_limbs(data + [P], MRR_N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)

    def cts():
        return np.stack([np.stack([rm.uniform_limbs(data, MRR_N) for _ in range(2)]) for _ in range(MRR_COUNT)])

    ca = torch.from_numpy(cts().view(np.int64)).to(dev)
    cb = torch.from_numpy(cts().view(np.int64)).to(dev)
    mrr_tune = autotune.tune_mul_relin_rescale(ctx, key, L, MRR_COUNT, reps=TUNE_REPS, warmup=3)
    out = torch.empty((MRR_COUNT, 2, L, MRR_N), dtype=torch.int64, device=dev)
    scratch = torch.empty(ctx.mrr_scratch_bytes(L, MRR_COUNT) // 8, dtype=torch.int64, device=dev)

    def mrr_batched():
        he.mul_relin_rescale(out, ca, cb, MRR_COUNT, key, ctx, L, scratch, stream=stream)

    ms_mrr = max_over_ranks(_time_steps(mrr_batched, args.steps, args.warmup, stream, barrier))
    mrr_dist = _distribution(_step_times(mrr_batched, max(20, args.steps), stream))
    s1 = scratch[: ctx.mrr_scratch_bytes(L, 1) // 8]

    def mrr_plain():
        for c in range(MRR_COUNT):
            he.mul_relin_rescale(out[c], ca[c], cb[c], 1, key, ctx, L, s1, stream=stream)

    ms_mrr_plain = max_over_ranks(_time_steps(mrr_plain, max(2, args.steps // 5), 3, stream, barrier))

    small = bench_small(args, stream, barrier) if "small" not in args.skip else None
    degrees = bench_degrees(args, stream, barrier) if "degrees" not in args.skip else None
    uneven = bench_uneven(args, stream, barrier) if "uneven" not in args.skip else None
    matrix = bench_matrix(args, stream, barrier) if "matrix" not in args.skip else None
    routines = bench_routines(args, stream, barrier) if "routines" not in args.skip else None
    encode = bench_encode(args, stream, barrier) if "encode" not in args.skip else None

    # end to end through host buffers: one he_ntt_host call per step (copy in,
    # forward, inverse, copy out, pipelined over chunks of 32 polynomials)
    back = torch.empty_like(pinned).pin_memory()
    work = torch.empty(4 * 32 * NTT_LIMBS * N, dtype=torch.int64, device=dev)

    def step_e2e():
        he.ntt_host(pinned, back, N, NTT_LIMBS, NTT_INSTANCES, tables,
                    he.NTT_OP_FORWARD | he.NTT_OP_INVERSE, work, stream=stream)

    # with the collector paused (as the serving loop runs): a full collection
    # of this process, which holds gigabytes of host data, can stall a step
    # for tens of milliseconds
    import gc
    gc.collect()
    gc.disable()
    try:
        ms_e2e = max_over_ranks(_time_steps(step_e2e, max(3, args.steps), max(3, args.warmup), stream, barrier))
    finally:
        gc.enable()
    torch.cuda.synchronize()
    assert torch.equal(back, pinned), "round trip changed the data"
    back.zero_()

    def step_serial():
        d.copy_(pinned, non_blocking=True)
        he.ntt_fwd(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        he.ntt_inv(d, N, NTT_LIMBS, NTT_INSTANCES, tables, stream=stream)
        back.copy_(d, non_blocking=True)

    ms_serial = max_over_ranks(_time_steps(step_serial, 3, 3, stream, barrier))

    # the host link alone: the same bytes copied in and out at the same time,
    # the floor of any step that moves them. Two forms, the faster counts:
    # the whole batch each way on two streams, and the chunks of the e2e
    # pipeline (32 polynomials, round-robin over four streams, each chunk
    # copied in then out on its stream) without the kernels; which of the
    # two the copy engines serve faster differs from box to box.
    s_out = torch.cuda.Stream()
    d2 = d.clone()   # holds the round-tripped batch, so `back` stays equal to the input

    def step_link():
        s_out.wait_stream(stream)
        with torch.cuda.stream(stream):
            d.copy_(pinned, non_blocking=True)
        with torch.cuda.stream(s_out):
            back.copy_(d2, non_blocking=True)
        stream.wait_stream(s_out)

    ms_link_whole = max_over_ranks(_time_steps(step_link, 3, 3, stream, barrier))
    link_streams = [torch.cuda.Stream() for _ in range(4)]
    chunk = 32

    def step_link_chunked():
        for ls in link_streams:
            ls.wait_stream(stream)
        for k, i in enumerate(range(0, NTT_INSTANCES, chunk)):
            with torch.cuda.stream(link_streams[k % 4]):
                d[i:i + chunk].copy_(pinned[i:i + chunk], non_blocking=True)
                back[i:i + chunk].copy_(d2[i:i + chunk], non_blocking=True)
        for ls in link_streams:
            stream.wait_stream(ls)

    ms_link_chunked = max_over_ranks(_time_steps(step_link_chunked, 3, 3, stream, barrier))
    ms_link = min(ms_link_whole, ms_link_chunked)
    del work, d2
    clk = clocks.stop()
    assert torch.equal(back, pinned), "round trip changed the data"
    del pinned, back
    serve = bench_serving(args) if "serving" not in args.skip else None

    # integer roof: register-resident butterflies on every SM
    sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device=dev)
    iters = 4096

    def probe():
        he.butterfly_probe(sink, sms * 8, 256, iters, stream=stream)

    ms_probe = _time_steps(probe, 5, 3, stream, lambda: None)
    bfly_rate = sms * 8 * 256 * 16 * iters / (ms_probe / 1e3)
    bfly_per_launch = limbs_total * (N // 2) * NTT_LOG_N

    peaks = _measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    # derived integer peak: the IMAD pipe fully busy at the sampled clock
    clock_hz = (clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0) * 1e6
    alu_peak = sms * clock_hz / FMAHEAVY_CYCLES_PER_BFLY

    def direction_roof(name, ms_dir, shape):
        gbs = bytes_per_launch / (ms_dir / 1e3) / 1e9
        bf = bfly_per_launch / (ms_dir / 1e3)
        key = (name, tuple(shape[:4]))
        return {"kernel": "k_ntt %s, 2^%d words per CTA x cluster of %d, 2^%d words per thread%s%s" % (
                    name, shape[0], N >> shape[0], shape[1], ", persistent" if shape[2] else "",
                    ", %d CTAs per SM" % shape[3] if len(shape) > 3 and shape[3] else ""),
                "ms": ms_dir, "achieved_tbfly": bf / 1e12, "alu_frac": bf / alu_peak,
                "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                "traffic": TRAFFIC.get(key)}

    roof_fwd = direction_roof("forward", fwd, tune["fwd"])
    roof_inv = direction_roof("inverse", inv, tune["inv"])
    dom = roof_inv if inv >= fwd else roof_fwd          # the larger share of the step
    bound_alu = dom["alu_frac"] >= dom["hbm_frac"]
    attach_rooflines(small, alu_peak, hbm_peak)
    attach_rooflines(degrees, alu_peak, hbm_peak)
    attach_rooflines(uneven, alu_peak, hbm_peak)
    attach_rooflines(matrix, alu_peak, hbm_peak)
    attach_rooflines(routines, alu_peak, hbm_peak)
    mrr_roof = roof_entry({k: v * MRR_COUNT for k, v in mrr_work(L + 1, MRR_N).items()}, ms_mrr / 1e3,
                          alu_peak, hbm_peak)
    value = job_value(world, 2 * limbs_total, ms)
    e2e_value = job_value(world, 2 * limbs_total, ms_e2e)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic: seeded uniform residues (SplitMix64), 60/50-bit NTT primes",
        "config": _ntt_config(f"replicas x{world}"),
        "ntt": {
            "batched_limbs_per_s": value,
            "graph_limbs_per_s": world * 2 * limbs_total / (ms_graph / 1e3),
            "plain_limbs_per_s": world * 2 * limbs_total / (ms_plain / 1e3),
            "naive_limbs_per_s": world * 2 * limbs_total / (ms_naive / 1e3),
            "fwd_limbs_per_s": world * limbs_total / (fwd / 1e3),
            "inv_limbs_per_s": world * limbs_total / (inv / 1e3),
            "fwd_ms": fwd, "inv_ms": inv, "speedup_vs_naive": ms_naive / ms,
            "step_distribution": step_dist,
        },
        "autotune": {"forward": dict(zip(("log_block", "log_thread_words", "persistent", "ctas_per_sm"), tune["fwd"])),
                     "inverse": dict(zip(("log_block", "log_thread_words", "persistent", "ctas_per_sm"), tune["inv"])),
                     "reps": TUNE_REPS,
                     "candidates": [{"shape": c["shape"], "ms_fwd": c.get("ms_fwd"), "ms_inv": c.get("ms_inv")}
                                    for c in tune["candidates"]]},
        "small_ntt": small,
        "ntt_by_degree": degrees,
        "uneven_batch": uneven,
        "matrix_mul_relin_rescale": matrix,
        "routines": routines,
        "encode_decode": encode,
        "serving": serve,
        "mul_relin_rescale": {
            "workload": "N=16384, data primes 60+6x50, special 60, 64 ciphertext pairs, level 6 -> 5",
            "batched_per_s": world * MRR_COUNT / (ms_mrr / 1e3),
            "plain_per_s": world * MRR_COUNT / (ms_mrr_plain / 1e3),
            "ms_per_batch": ms_mrr,
            "batch_distribution": mrr_dist,
            "transforms_per_op": (L + 1) ** 2 + 5 * (L + 1) + 2,
            "work_per_op": mrr_work(L + 1, MRR_N),
            "roofline": mrr_roof,
            "autotune": mrr_tune,
        },
        "roofline": {
            "kernel": dom["kernel"],
            "bound": "alu" if bound_alu else "hbm",
            "achieved": dom["achieved_tbfly"] if bound_alu else dom["achieved_gbs"],
            "peak": alu_peak / 1e12 if bound_alu else hbm_peak,
            "unit": "Tbutterfly/s" if bound_alu else "GB/s",
            "frac": dom["alu_frac"] if bound_alu else dom["hbm_frac"],
            "traffic": dom["traffic"],
            "dominant": "inverse" if dom is roof_inv else "forward",
            "directions": {"forward": roof_fwd, "inverse": roof_inv},
            "hbm": {"achieved_gbs": dom["achieved_gbs"], "peak_gbs": hbm_peak, "frac": dom["hbm_frac"],
                    "peak_source": "measured copy bandwidth" if peaks.get("hbm_gbs") else "fallback"},
            "alu": {"achieved_tbfly": dom["achieved_tbfly"], "peak_tbfly": alu_peak / 1e12, "frac": dom["alu_frac"],
                    "peak_source": f"derived: {sms} SMs x {clock_hz / 1e6:.0f} MHz / "
                                   f"{FMAHEAVY_CYCLES_PER_BFLY} IMAD-pipe cycles per butterfly",
                    "probe_tbfly": bfly_rate / 1e12, "frac_of_probe": dom["achieved_tbfly"] * 1e12 / bfly_rate,
                    "probe_source": "register-resident butterfly probe, same run"},
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "butterflies_per_launch": bfly_per_launch,
        },
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * limbs_total * N,
                "d2h_bytes_per_step": 8 * limbs_total * N, "ms_per_step": ms_e2e,
                "call": "he_ntt_host(forward | inverse), pinned host buffers, 4 streams x 32-polynomial chunks",
                "whole_batch_copies_value": world * 2 * limbs_total / (ms_serial / 1e3),
                "host_link": {"ms_copy_in_and_out": ms_link, "ms_whole_batch_copies": ms_link_whole,
                              "ms_chunked_copies": ms_link_chunked,
                              "gbs_per_direction": 8 * limbs_total * N / (ms_link / 1e3) / 1e9,
                              "e2e_frac_of_link_bound": ms_link / ms_e2e}},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------ other workloads

def bench_degrees(args, stream, barrier):
    """The batched transform at every supported degree, N = 2^10 .. 2^16:
    polynomials of 8 limbs (four 60-bit and four 50-bit primes), as many as
    make 2^25 words (256 MiB per direction, larger than L2), forward then
    inverse in place, one launch per direction, the shapes the autotuner
    picks for this batch (2^15 keeps those it picked for the headline batch,
    which the later sections run). Inputs are uniform residues drawn on the
    device (the timing does not depend on them; the GPU tests check every
    degree against the oracle)."""
    import torch

    from paper_2109_14704_gb300 import autotune, he

    limbs, words = 8, 1 << 25
    rows = []
    for log_n in range(10, 17):
        N = 1 << log_n
        qs = he.primes_generate(60, 2 * N, 4) + he.primes_generate(50, 2 * N, 4)
        tables = he.NttTables(N, qs)
        count = words // (limbs * N)
        tuned = None
        if log_n != NTT_LOG_N:
            tuned = autotune.tune_uniform(N, limbs, count, moduli=qs, reps=TUNE_REPS, warmup=3,
                                          cache_path=None if args.no_tune_cache else autotune.DEFAULT_CACHE)
        g = torch.Generator(device="cuda")
        g.manual_seed(log_n)
        d = torch.randint(0, 1 << 62, (count, limbs, N), dtype=torch.int64, device="cuda", generator=g)
        d %= torch.tensor(qs, dtype=torch.int64, device="cuda").view(1, limbs, 1)
        fwd_ms, inv_ms = [], []
        for it in range(8):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            he.ntt_fwd(d, N, limbs, count, tables, stream=stream)
            e[1].record(stream)
            he.ntt_inv(d, N, limbs, count, tables, stream=stream)
            e[2].record(stream)
            torch.cuda.synchronize()
            if it >= 3:
                fwd_ms.append(e[0].elapsed_time(e[1]))
                inv_ms.append(e[1].elapsed_time(e[2]))
        fwd, inv = statistics.median(fwd_ms), statistics.median(inv_ms)
        items = count * limbs
        rows.append({"N": N, "polys": count, "limbs": items,
                     "shape": ({"forward": list(tuned["fwd"]), "inverse": list(tuned["inv"])} if tuned
                               else "the headline batch's tuned shape"),
                     "fwd_ms": fwd, "inv_ms": inv, "limbs_per_s": 2 * items / ((fwd + inv) / 1e3),
                     "_work": {"bfly": 2 * items * (N // 2) * log_n, "bytes": 2 * 16 * N * items,
                               "seconds": (fwd + inv) / 1e3}})
        del d, tables
    return {"workload": "batched forward + inverse, 8 limbs per polynomial, 2^25 words per direction, "
                        "N = 2^10 .. 2^16, shapes tuned per degree", "degrees": rows}


def bench_small(args, stream, barrier):
    """The plain single transform (N = 4096, two 60-bit primes, two
    polynomials a and b): latency of forward + inverse, and of the
    negacyclic product a b = INTT(NTT(a) . NTT(b)), each a short chain of
    launches on one stream (latency bound: reported in microseconds)."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    N, limbs = 4096, 2
    qs = he.primes_generate(60, 2 * N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(1)
    a = torch.from_numpy(np.stack([r.uniform_limbs(qs, N)]).view(np.int64)).cuda()
    b = torch.from_numpy(np.stack([r.uniform_limbs(qs, N)]).view(np.int64)).cuda()
    c = torch.empty_like(a)

    def fwd_inv():
        he.ntt_fwd(a, N, limbs, 1, tables, stream=stream)
        he.ntt_inv(a, N, limbs, 1, tables, stream=stream)

    a2, b2, c2 = a.clone(), b.clone(), torch.empty_like(a)

    def product():
        # forward, forward, dyadic, inverse on copies, in place (their
        # contents drift from step to step, which does not change the work)
        he.ntt_fwd(a2, N, limbs, 1, tables, stream=stream)
        he.ntt_fwd(b2, N, limbs, 1, tables, stream=stream)
        he.dyadic_mul(c2, a2, b2, N, limbs, 1, tables, stream=stream)
        he.ntt_inv(c2, N, limbs, 1, tables, stream=stream)

    def fused():
        he.negacyclic_mul(c, a, b, N, limbs, 1, tables, stream=stream)

    reps = 200
    us_fi = _time_steps(fwd_inv, reps, 20, stream, barrier) * 1e3
    us_prod = _time_steps(product, reps, 20, stream, barrier) * 1e3
    us_fused = _time_steps(fused, reps, 20, stream, barrier) * 1e3

    # the same product over a batch that does not fit in L2: 128 polynomials
    # x 8 limbs at N = 2^15 (3 x 256 MiB), fused (one launch: 24 B per word
    # through HBM) against forward, forward, dyadic, inverse (72 B per word)
    Nb, lb, cb = 32768, 8, 128
    qb = he.primes_generate(60, 2 * Nb, 4) + he.primes_generate(50, 2 * Nb, 4)
    tb = he.NttTables(Nb, qb)
    A = torch.from_numpy(np.stack([r.uniform_limbs(qb, Nb) for _ in range(cb)]).view(np.int64)).cuda()
    B = torch.from_numpy(np.stack([r.uniform_limbs(qb, Nb) for _ in range(cb)]).view(np.int64)).cuda()
    Cb = torch.empty_like(A)

    def batch_fused():
        he.negacyclic_mul(Cb, A, B, Nb, lb, cb, tb, stream=stream)

    A2, B2, C2 = A.clone(), B.clone(), torch.empty_like(A)

    def batch_unfused():
        # the same four passes on copies, in place (their contents drift
        # from step to step, which does not change the work)
        he.ntt_fwd(A2, Nb, lb, cb, tb, stream=stream)
        he.ntt_fwd(B2, Nb, lb, cb, tb, stream=stream)
        he.dyadic_mul(C2, A2, B2, Nb, lb, cb, tb, stream=stream)
        he.ntt_inv(C2, Nb, lb, cb, tb, stream=stream)

    steps = max(3, args.steps // 2)
    ms_f = _time_steps(batch_fused, steps, 3, stream, barrier)
    ms_u = _time_steps(batch_unfused, steps, 3, stream, barrier)
    limbs_b = lb * cb
    bfly = 3 * limbs_b * (Nb // 2) * 15
    return {"workload": "N=4096, 2 x 60-bit primes, one polynomial (forward + inverse) or two (product)",
            "us_forward_inverse": us_fi, "us_negacyclic_product": us_prod, "us_negacyclic_product_fused": us_fused,
            "launches": {"forward_inverse": 2, "product": 4, "product_fused": 1},
            "note": "latency of back-to-back launches on one stream (inputs in L2)",
            "batch": {"workload": "negacyclic product, 128 polys x 8 limbs at N=2^15",
                      "_work": {"bfly": bfly, "products": limbs_b * Nb, "bytes": 24 * Nb * limbs_b,
                                "seconds": ms_f / 1e3},
                      "ms_fused": ms_f, "fused_products_per_s": limbs_b / (ms_f / 1e3),
                      "fused_tbfly_per_s": bfly / (ms_f / 1e3) / 1e12,
                      "ms_unfused": ms_u, "unfused_products_per_s": limbs_b / (ms_u / 1e3)}}


def bench_uneven(args, stream, barrier):
    """Uneven batch: 512 polynomials, N uniform in {2^12 .. 2^15}, 1-16 limbs
    each from a pool of sixteen 50-60-bit primes = 1 mod 2^16 (seed 3). One
    mixed-degree launch per direction versus per-degree launches (one cluster
    per limb) versus one launch per polynomial."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    pool = he.primes_generate(60, 1 << 16, 6) + he.primes_generate(55, 1 << 16, 5) + \
        he.primes_generate(50, 1 << 16, 5)
    degrees = [4096, 8192, 16384, 32768]
    tables = {N: he.NttTables(N, pool) for N in degrees}
    r = Rng(3)
    Ns = r.choice(degrees, 512)
    Ls = r.choice(list(range(1, 17)), 512)
    Fs = [int(x) for x in r.choice(list(range(16)), 512)]
    Fs = [min(f, 16 - L) for f, L in zip(Fs, Ls)]
    polys = [torch.from_numpy(r.uniform_limbs(pool[f:f + L], N).view(np.int64)).cuda()
             for N, L, f in zip(Ns, Ls, Fs)]
    entries = [(polys[i], tables[N], N, L, f) for i, (N, L, f) in enumerate(zip(Ns, Ls, Fs))]
    limbs = sum(Ls)
    words = sum(N * L for N, L in zip(Ns, Ls))
    mixed = he.NttPlan(entries)
    per_degree = he.NttPlan(entries, shapes={N: he.ntt_shapes(N)[0][:2] for N in degrees})

    def run_plan(plan):
        def step():
            plan.fwd(stream=stream)
            plan.inv(stream=stream)
        return step

    singles = [he.NttPlan([e]) for e in entries]     # one launch per polynomial

    def step_plain():
        for pl in singles:
            pl.fwd(stream=stream)
        for pl in singles:
            pl.inv(stream=stream)

    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        mixed.fwd(stream=side)
        mixed.inv(stream=side)
        with torch.cuda.graph(g, stream=side):
            mixed.fwd(stream=side)
            mixed.inv(stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    ms_mixed = _time_steps(run_plan(mixed), args.steps, args.warmup, stream, barrier)
    ms_graph = _time_steps(g.replay, args.steps, args.warmup, stream, barrier)
    ms_deg = _time_steps(run_plan(per_degree), args.steps, args.warmup, stream, barrier)
    ms_plain = _time_steps(step_plain, max(2, args.steps // 5), 3, stream, barrier)
    bfly = sum(L * (N // 2) * (N.bit_length() - 1) for N, L in zip(Ns, Ls))
    work = {"bfly": 2 * bfly, "products": 0, "bytes": 2 * 16 * words}      # forward + inverse per step
    return {
        "workload": "512 polys, N in {4096..32768}, 1-16 limbs of 50-60-bit primes, seed 3",
        "limbs": limbs, "words": words,
        "mixed": {"_work": dict(work, seconds=ms_mixed / 1e3)},
        "per_degree": {"_work": dict(work, seconds=ms_deg / 1e3)},
        "mixed_single_launch_limbs_per_s": 2 * limbs / (ms_mixed / 1e3),
        "mixed_graph_limbs_per_s": 2 * limbs / (ms_graph / 1e3),
        "per_degree_launches_limbs_per_s": 2 * limbs / (ms_deg / 1e3),
        "plain_per_poly_limbs_per_s": 2 * limbs / (ms_plain / 1e3),
        "mixed_gbs": 2 * 16 * words / (ms_mixed / 1e3) / 1e9,
        "launches_per_direction": {"mixed": mixed.launches, "per_degree": per_degree.launches,
                                   "plain": len(singles)},
    }


def bench_matrix(args, stream, barrier):
    """Element-wise product of two 32 x 32 matrices of ciphertexts: 1024
    MulLinRS at N = 8192, data primes 60/40/40, special prime 60, one call;
    and the encrypted matrix product C += A B (32x32x32 and the paper's
    100x100x1 and 10x9x8) at the same parameters."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    N, count = 8192, 1024
    data, P = he.chain_primes(N, [60, 40, 40], 60)
    ctx = he.Context(N, data, P)
    L = 2
    r = Rng(4)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(3)])
    key = he.RelinKey(ctx, evk)
    mk = lambda: torch.from_numpy(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])
                                            for _ in range(count)]).view(np.int64)).cuda()
    A, B = mk(), mk()
    out = torch.empty((count, 2, L, N), dtype=torch.int64, device="cuda")
    scratch = torch.empty(ctx.mrr_scratch_bytes(L, count) // 8, dtype=torch.int64, device="cuda")
    from paper_2109_14704_gb300 import autotune
    tune = autotune.tune_mul_relin_rescale(ctx, key, L, count, reps=TUNE_REPS, warmup=3)

    def step():
        he.mul_relin_rescale(out, A, B, count, key, ctx, L, scratch, stream=stream)

    ms = _time_steps(step, args.steps, args.warmup, stream, barrier)
    res = {"workload": "32x32 element-wise, N=8192, primes 60/40/40 + 60, 1024 MulLinRS per step",
           "ms_per_step": ms, "mul_relin_rescale_per_s": count / (ms / 1e3),
           "_work": dict({k: v * count for k, v in mrr_work(L + 1, N).items()}, seconds=ms / 1e3),
           "eval_log_thread_words": tune["log_thread_words"]}
    del A, B, out, scratch
    # the encrypted matrix product C += A B (matMul_mxnxk): tensors
    # accumulated over k, one relin + rescale per output, add into C
    res["matmul"] = {}
    for (m, k, n) in ((32, 32, 32), (100, 100, 1), (10, 9, 8)):
        Am = torch.from_numpy(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])
                                        for _ in range(m * k)]).view(np.int64)).cuda()
        Bm = torch.from_numpy(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])
                                        for _ in range(k * n)]).view(np.int64)).cuda()
        Cm = torch.from_numpy(np.stack([np.stack([r.uniform_limbs(data[:L], N) for _ in range(2)])
                                        for _ in range(m * n)]).view(np.int64)).cuda()
        T = torch.empty((m * n, 3, L + 1, N), dtype=torch.int64, device="cuda")
        R = torch.empty((m * n, 2, L, N), dtype=torch.int64, device="cuda")
        sc = torch.empty(ctx.mrr_scratch_bytes(L, m * n) // 8, dtype=torch.int64, device="cuda")

        def t_step():
            he.ct_matmul_tensor(T, Am, Bm, m, k, n, ctx, L, stream=stream)

        def mm_step():
            t_step()
            he.relin_rescale(R, T, m * n, key, ctx, L, sc, stream=stream)
            he.ct_add(Cm, Cm, R, m * n, 2, ctx, L - 1, stream=stream)

        ms_t = _time_steps(t_step, max(3, args.steps // 2), 3, stream, barrier)
        ms_mm = _time_steps(mm_step, max(3, args.steps // 2), 3, stream, barrier)
        res["matmul"][f"{m}x{k}x{n}"] = {
            "ms_per_matmul": ms_mm, "ms_tensor": ms_t, "tensor_products": m * k * n,
            "relin_rescale_outputs": m * n,
            "tensor_products_per_s": m * k * n / (ms_t / 1e3)}
        del Am, Bm, Cm, T, R, sc
    return res


def bench_routines(args, stream, barrier):
    """The paper's five-routine set at its size (Sec. IV-C: N = 32K, 8 RNS
    limbs; here data primes 60 + 7 x 50, special prime 60, level 7), batches
    of 16 ciphertexts: MulLin, MulLinRS, SqrLinRS, Rotate (k = 1)."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    N, count = 32768, 16
    data, P = he.chain_primes(N, [60] + [50] * 7, 60)
    ctx = he.Context(N, data, P)
    L = len(data) - 1
    r = Rng(8)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)          # also serves as a (pseudo-random) Galois key for timing
    mk = lambda: torch.from_numpy(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])
                                            for _ in range(count)]).view(np.int64)).cuda()
    A, B = mk(), mk()
    out_l = torch.empty((count, 2, L + 1, N), dtype=torch.int64, device="cuda")
    out_r = torch.empty((count, 2, L, N), dtype=torch.int64, device="cuda")
    sc = torch.empty(max(ctx.mrr_scratch_bytes(L, count), ctx.rotate_scratch_bytes(L, count)) // 8,
                     dtype=torch.int64, device="cuda")
    g = pow(5, 1, 2 * N)
    ops = {
        "mul_lin": lambda: he.mul_relin(out_l, A, B, count, key, ctx, L, sc, stream=stream),
        "mul_lin_rs": lambda: he.mul_relin_rescale(out_r, A, B, count, key, ctx, L, sc, stream=stream),
        "sqr_lin_rs": lambda: he.sqr_relin_rescale(out_r, A, count, key, ctx, L, sc, stream=stream),
        "rotate": lambda: he.rotate(out_l, A, count, g, key, ctx, L, sc, stream=stream),
    }
    res = {"workload": f"N=32768, {len(data)} data primes (60 + 7 x 50) + 60-bit special, level {L}, "
                       f"batches of {count} ciphertexts"}
    for name, fn in ops.items():
        ms = _time_steps(fn, max(3, args.steps // 2), 3, stream, barrier)
        res[name] = {"ms_per_batch": ms, "per_s": count / (ms / 1e3)}
        if name in ("mul_lin_rs", "sqr_lin_rs"):
            res[name]["_work"] = dict({k: v * count for k, v in mrr_work(L + 1, N).items()}, seconds=ms / 1e3)
    return res


def bench_encode(args, stream, barrier):
    """Device Encode / Decode (Sec. II-A) at the routine-set size: N = 2^15,
    level 7 (8 limbs: 60 + 7 x 50 bits), batches of 64 messages of 16384
    complex slots (scale 2^40). The components that the library exposes are
    timed alone: the CRT lift of decoding, and the NTTs of the same limbs;
    the FP64 probe gives the rate that bounds the slot FFT."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    N, count, level, scale = 32768, 64, 7, 2.0 ** 40
    n = N // 2
    data, P = he.chain_primes(N, [60] + [50] * 7, 60)
    ctx = he.Context(N, data, P)
    enc = he.Encoder(ctx)
    tables = he.NttTables(N, data)
    r = Rng(9)
    z = torch.from_numpy(np.stack([r.complex_slots(n) for _ in range(count)])).cuda()
    zo = torch.empty_like(z)
    pt = torch.empty((count, level + 1, N), dtype=torch.int64, device="cuda")
    coef = torch.empty_like(pt)
    m = torch.empty((count, N), dtype=torch.float64, device="cuda")
    sc = torch.empty(max(enc.encode_scratch_bytes(count), enc.decode_scratch_bytes(level, count)) // 8,
                     dtype=torch.int64, device="cuda")
    steps = max(3, args.steps // 2)
    ms_enc = _time_steps(lambda: enc.encode(pt, z, count, scale, level, sc, stream=stream), steps, 3, stream, barrier)
    ms_dec = _time_steps(lambda: enc.decode(zo, pt, count, scale, level, sc, stream=stream), steps, 3, stream,
                         barrier)
    torch.cuda.synchronize()
    err = float(((zo - z).abs().max() / z.abs().max()).item())
    coef.copy_(pt)
    ms_crt = _time_steps(lambda: enc.crt_compose(m, coef, count, level, stream=stream), steps, 3, stream, barrier)
    ms_fwd = _time_steps(lambda: he.ntt_fwd(coef, N, level + 1, count, tables, stream=stream), steps, 3, stream,
                         barrier)
    ms_inv = _time_steps(lambda: he.ntt_inv(coef, N, level + 1, count, tables, stream=stream), steps, 3, stream,
                         barrier)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    iters = 4096
    ms_probe = _time_steps(lambda: he.fp64_probe(sink, sms * 8, 256, iters, stream=stream), 5, 3, stream, barrier)
    fp64_peak = sms * 8 * 256 * iters * 16 / (ms_probe / 1e3) / 1e12
    fft_flop = 5.0 * n * math.log2(n) * count
    ms_fft_enc = ms_enc - ms_fwd
    return {
        "workload": f"N=32768, level {level} ({level + 1} limbs: 60 + 7 x 50 bits), {count} messages of {n} "
                    "complex slots, scale 2^40",
        "encode": {"ms_per_batch": ms_enc, "per_s": count / (ms_enc / 1e3)},
        "decode": {"ms_per_batch": ms_dec, "per_s": count / (ms_dec / 1e3)},
        "round_trip_max_rel_err": err,
        "components_ms": {"ntt_fwd": ms_fwd, "ntt_inv": ms_inv, "crt_lift": ms_crt,
                          "encode_minus_ntt": ms_fft_enc, "decode_minus_intt_crt": ms_dec - ms_inv - ms_crt},
        "fp64": {"probe_tflops": fp64_peak,
                 "encode_fft_tflops": fft_flop / (ms_fft_enc / 1e3) / 1e12,
                 "fft_flop_per_batch": fft_flop},
    }


SERVE_WARMUP = 1000
SERVE_POOL = 4          # input pairs per (N, level) bucket: about 1.1 GB of pinned host ciphertexts in all
SERVE_SWEEP = (1000.0, 4000.0, 8000.0, 16000.0)


def bench_serving(args):
    """Poisson arrivals at 2000 requests/s of MulLinRS jobs, N in {8192,
    16384, 32768}, levels 2-16, keys resident, 64 GB admission budget: the
    continuous-batching server (batches per degree and level), the same
    server batching every level of a degree together (mixed-level batches,
    one launch per pipeline stage), batching every degree and level together
    (multi-degree batches, one launch per pipeline stage), and the server
    with one request per launch (one slot, one stream). Each server reserves its buffer pool at
    start-up (prewarm) and runs its loop without collector pauses. Every
    measured run follows SERVE_WARMUP warm-up requests; requests draw their
    inputs from SERVE_POOL pinned host pairs per bucket (uploaded per
    request). A short sweep of the arrival rate up to saturation shows where
    batching pays."""
    from paper_2109_14704_gb300 import serving

    import torch

    out = {"workload": f"Poisson 2000 req/s, N in {{8192,16384,32768}}, levels 2-16, budget 64 GB, "
                       f"{args.serve_requests} requests after {SERVE_WARMUP} warm-up, {SERVE_POOL} input pairs "
                       f"per (N, level) bucket"}
    sweep_n = max(1000, args.serve_requests // 5)
    pool = None
    for name, kw in (("batched", dict(slots=16, streams=4, prewarm_batches=8)),
                     ("mixed_levels", dict(slots=16, streams=4, prewarm_batches=8, mixed_levels=True)),
                     ("mixed_degrees", dict(slots=16, streams=4, prewarm_batches=8, mixed_degrees=True)),
                     ("plain", dict(slots=1, streams=1, prewarm_batches=4))):
        # every server starts from an empty allocator cache (the previous
        # phases' freed blocks would otherwise count against device memory)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        srv = serving.Server(pool_per_bucket=SERVE_POOL, seed=5, pool=pool, **kw)
        pool = srv.pool                      # generated once, shared by the three servers
        srv.run(srv.make_requests(SERVE_WARMUP, rate=2000.0, seed=55))     # warm-up
        srv.completed.clear()
        srv.batches_launched = 0
        out[name] = srv.run(srv.make_requests(args.serve_requests, rate=2000.0, seed=5))
        out[name]["input_pool_gb"] = sum(t.numel() * 8 for t in srv.pool.values()) / 2 ** 30
        # capacity: the same request mix arriving far faster than it can be served
        srv.completed.clear()
        srv.batches_launched = 0
        sat = srv.run(srv.make_requests(args.serve_requests, rate=1e6, seed=6))
        out[name]["saturated_throughput_per_s"] = sat["throughput_per_s"]
        out[name]["saturated_mean_batch"] = sat["mean_batch"]
        out[name]["expand_group"] = srv.expand_group
        sw = []
        for rate in SERVE_SWEEP:
            srv.completed.clear()
            srv.batches_launched = 0
            r = srv.run(srv.make_requests(sweep_n, rate=rate, seed=7))
            sw.append({"rate": rate, "requests": sweep_n, "throughput_per_s": r["throughput_per_s"],
                       "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "mean_batch": r["mean_batch"]})
        out[name]["rate_sweep"] = sw
        del srv
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- CPU oracle

def _ntt_config(parallelism: str) -> dict:
    N = 1 << NTT_LOG_N
    return {"workload": "NTT N=2^15, 1024 instances x 8 RNS limbs (4 x 60-bit, 4 x 50-bit primes), "
                        "forward + inverse per step, in place",
            "N": N, "limbs": NTT_LIMBS, "instances": NTT_INSTANCES, "parallelism": parallelism,
            "l2": "inputs larger than L2 (2 GiB per direction)"}


def cpu_baseline(target_seconds: float, limbs: int | None = None) -> dict:
    """The oracle's forward + inverse NTT at N = 2^15 on a bounded sample of
    the workload's limbs, on all host cores: the median of CPU_RUNS runs,
    each about target_seconds / CPU_RUNS of CPU work."""
    import numpy as np

    import oracle
    from paper_2109_14704_gb300.synth import Rng

    N = 1 << NTT_LOG_N
    qs = _ntt_moduli(cpu_oracle=True)
    cores = os.cpu_count() or 1
    x = np.stack([Rng(3000).uniform_limbs(qs, N)])
    singles = []
    for _ in range(3):                                  # calibrate on one thread
        t = time.perf_counter()
        y = oracle.ntt_fwd_many(x, qs, 1)
        oracle.ntt_inv_many(y, qs, 1)
        singles.append((time.perf_counter() - t) / (2 * NTT_LIMBS))
    per_transform = statistics.median(singles)
    if limbs is None:
        polys = max(1, int(target_seconds / CPU_RUNS * cores / (per_transform * 2 * NTT_LIMBS)))
    else:
        polys = max(1, limbs // NTT_LIMBS)
    polys = min(polys, NTT_INSTANCES)
    r = Rng(3001)
    x = np.stack([r.uniform_limbs(qs, N) for _ in range(polys)])
    walls = []
    for _ in range(CPU_RUNS):
        t = time.perf_counter()
        y = oracle.ntt_fwd_many(x, qs, cores)
        z = oracle.ntt_inv_many(y, qs, cores)
        walls.append(time.perf_counter() - t)
        assert np.array_equal(z, x)
    wall = statistics.median(walls)
    transforms = 2 * polys * NTT_LIMBS
    return {"value": transforms / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": 1.0 / per_transform,
            "runs": CPU_RUNS, "wall_s": walls,
            "sample": f"{polys} of {NTT_INSTANCES} instances x {NTT_LIMBS} limbs at N=2^15, forward + inverse "
                      f"({transforms} limb transforms per run, median of {CPU_RUNS} runs, {wall:.2f} s each; "
                      f"plain __int128 % oracle built with gcc -O3, one host thread per (instance, limb) "
                      f"unit on {cores} cores); single_thread_value: one instance ({2 * NTT_LIMBS} limb "
                      f"transforms) on one thread, median of 3"}


def run_reference(args, rank, world):
    """The oracle on the headline workload: each step is the forward and the
    inverse transform of REF_INSTANCES of the 1024 instances (all 8 limbs),
    on all host cores."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2109_14704_gb300.synth import Rng

    N = 1 << NTT_LOG_N
    qs = _ntt_moduli(cpu_oracle=True)
    cores = os.cpu_count() or 1
    polys = getattr(args, "ref_instances", REF_INSTANCES)
    r = Rng(4000)
    x = np.stack([r.uniform_limbs(qs, N) for _ in range(polys)])

    def step():
        y = oracle.ntt_fwd_many(x, qs, cores)
        oracle.ntt_inv_many(y, qs, cores)

    for _ in range(args.warmup):
        step()
    walls = []
    for _ in range(args.steps):
        t = time.perf_counter()
        step()
        walls.append(time.perf_counter() - t)
    wall = sum(walls) / len(walls)
    transforms = 2 * polys * NTT_LIMBS
    value = transforms / wall
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic: seeded uniform residues (SplitMix64), 60/50-bit NTT primes",
        "config": _ntt_config("replicas x1"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{polys} of {NTT_INSTANCES} instances (1/{NTT_INSTANCES // polys} of the batch) "
                                   f"x {NTT_LIMBS} limbs per step, forward + inverse, plain __int128 % oracle "
                                   f"(gcc -O3), one host thread per (instance, limb) unit; median step "
                                   f"{statistics.median(walls):.2f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_case(args):
    """A small case of one kernel family: `ntt` transforms args.instances x 8
    limbs at N = 2^15 (64 instances = 128 MiB, above the L2 size) forward
    then inverse, `mrr` runs one MulLinRS batch of args.instances pairs on
    the CKKS workload (--shape: log2 words per thread of its kernels),
    `encode` encodes and decodes args.instances messages at N = 2^15 with 8
    limbs, `product` runs the fused negacyclic product of args.instances x 8
    limbs at N = 2^15, `probe` the butterfly probe. Each runs `--steps`
    times."""
    import numpy as np
    import torch

    from paper_2109_14704_gb300 import he
    from paper_2109_14704_gb300.synth import Rng

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    he.load()
    if args.profile_case == "ntt":
        N = 1 << NTT_LOG_N
        qs = _ntt_moduli()
        tables = he.NttTables(N, qs)
        if args.shape:   # "lb,le[,persistent]" for both directions, or "fwd/inv"
            parts = args.shape.split("/")
            for direction, spec in zip((he.FORWARD, he.INVERSE), parts if len(parts) == 2 else parts * 2):
                he.ntt_set_shape(N, *([int(v) for v in spec.split(",")] + [0, 0, 0])[:3], direction=direction)
        r = Rng(1)
        d = torch.from_numpy(np.stack([r.uniform_limbs(qs, N) for _ in range(args.instances)]).view(np.int64)).to(dev)
        for _ in range(args.steps):
            he.ntt_fwd(d, N, NTT_LIMBS, args.instances, tables)
            he.ntt_inv(d, N, NTT_LIMBS, args.instances, tables)
    elif args.profile_case == "mrr":
        data, P = he.chain_primes(MRR_N, MRR_BITS, 60)
        ctx = he.Context(MRR_N, data, P)
        L, count = len(data) - 1, args.instances
        rm = Rng(2)
        evk = np.stack([np.stack([rm.uniform_limbs(data + [P], MRR_N) for _ in range(2)]) for _ in range(len(data))])
        key = he.RelinKey(ctx, evk)
        mk = lambda: torch.from_numpy(np.stack([np.stack([rm.uniform_limbs(data, MRR_N) for _ in range(2)])
                                                 for _ in range(count)]).view(np.int64)).to(dev)
        ca, cb = mk(), mk()
        out = torch.empty((count, 2, L, MRR_N), dtype=torch.int64, device=dev)
        scratch = torch.empty(ctx.mrr_scratch_bytes(L, count) // 8, dtype=torch.int64, device=dev)
        if args.shape:   # words per thread of the evaluation kernels, as log2
            ctx.set_eval_shape(int(args.shape))
        for _ in range(args.steps):
            he.mul_relin_rescale(out, ca, cb, count, key, ctx, L, scratch)
    elif args.profile_case == "mrr_multi":
        # the serving mix as one multi-degree batch: 16 jobs, N cycling over
        # 2^13, 2^14, 2^15, levels drawn from 2..16, args.instances pairs each
        rm = Rng(3)
        ctxs, keys = {}, {}
        for N in (8192, 16384, 32768):
            data, P = he.chain_primes(N, [60] + [50] * 16, 60)
            ctxs[N] = he.Context(N, data, P)
            evk = np.stack([np.stack([rm.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(17)])
            keys[N] = he.RelinKey(ctxs[N], evk)
        levels = [int(v) for v in rm.choice(list(range(2, 17)), 16)]
        jobs = []
        for j, lv in enumerate(levels):
            N = (8192, 16384, 32768)[j % 3]
            ctx = ctxs[N]
            qs = ctx.data_moduli[:lv + 1]
            mk = lambda: torch.from_numpy(np.stack([np.stack([rm.uniform_limbs(qs, N) for _ in range(2)])
                                                     for _ in range(args.instances)]).view(np.int64)).to(dev)
            out = torch.empty((args.instances, 2, lv, N), dtype=torch.int64, device=dev)
            jobs.append((out, mk(), mk(), args.instances, lv, keys[N], ctx))
        scratch = torch.empty(he.mul_relin_rescale_multi_scratch_bytes([(j[3], j[4], j[5], j[6]) for j in jobs]) // 8,
                              dtype=torch.int64, device=dev)
        for _ in range(args.steps):
            he.mul_relin_rescale_multi(jobs, scratch)
    elif args.profile_case == "product":
        N = 1 << NTT_LOG_N
        qs = _ntt_moduli()
        tables = he.NttTables(N, qs)
        r = Rng(6)
        mk = lambda: torch.from_numpy(np.stack([r.uniform_limbs(qs, N) for _ in range(args.instances)])
                                      .view(np.int64)).to(dev)
        a, b = mk(), mk()
        c = torch.empty_like(a)
        for _ in range(args.steps):
            he.negacyclic_mul(c, a, b, N, NTT_LIMBS, args.instances, tables)
    elif args.profile_case == "encode":
        N, level = 32768, 7
        data, P = he.chain_primes(N, [60] + [50] * 7, 60)
        enc = he.Encoder(he.Context(N, data, P))
        count = args.instances
        r = Rng(9)
        z = torch.from_numpy(np.stack([r.complex_slots(N // 2) for _ in range(count)])).to(dev)
        zo = torch.empty_like(z)
        pt = torch.empty((count, level + 1, N), dtype=torch.int64, device=dev)
        sc = torch.empty(enc.decode_scratch_bytes(level, count) // 8, dtype=torch.int64, device=dev)
        for _ in range(args.steps):
            enc.encode(pt, z, count, 2.0 ** 40, level, sc)
            enc.decode(zo, pt, count, 2.0 ** 40, level, sc)
    else:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device=dev)
        for _ in range(args.steps):
            he.butterfly_probe(sink, sms * 8, 256, 1024)
    torch.cuda.synchronize()
    print(f"profile case {args.profile_case}: done")


def main():
    args = _args()
    rank, world, local = _dist()
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Throughput of the whole hot path -- phase one (2-bit encode, minimizers, super-mer bins)
plus phase two (extract, canonicalise, count, overflow, compact + min-count filter) -- in
canonical k-mers counted per second on one B300, bit-exact integer counts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = gerbil_partition + gerbil_count_batch over all bins of one synthetic read set that
is already resident in HBM.  Under torchrun each rank runs an independent replica (the path
has no exchange step); the value is the k-mers of all ranks over the slowest rank's time.
Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("canonical k-mers counted/sec on 1 B300 (bit-exact), fraction of HBM roofline; "
          "batched vs per-bin")
UNIT = "k-mers/s"
DEFAULT_WORKLOAD = "genome5M-30x-k65"
SERVING_WORKLOAD = "serving-poisson20-k32-65-127"
L2_BYTES = 126 * 2 ** 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=80)
    ap.add_argument("--e2e-workers", type=int, default=4,
                    help="host threads (one context and stream each) driving the e2e steps")
    ap.add_argument("--per-bin-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-windows", type=int, default=3_500_000,
                    help="k-mer windows of the oracle's timed sample (cpu_baseline)")
    ap.add_argument("--ref-sample-windows", type=int, default=400_000,
                    help="k-mer windows per step of --impl reference")
    ap.add_argument("--fused", type=int, default=None,
                    help="phase-two form: 0 all tables, 1 fused queue kernel, 2 waves")
    ap.add_argument("--schedule", type=int, default=None, help="1 device queue, 0 fixed striding")
    ap.add_argument("--autotune", action="store_true",
                    help="form, schedule and per-class load factors from the autotuner")
    ap.add_argument("--graph", action="store_true", help="phase two as one captured CUDA graph")
    ap.add_argument("--probe-scheme", type=int, default=None,
                    help="0 linear probing (default), 1 windowed double hashing (Sec. 3.3)")
    ap.add_argument("--claim-first", type=int, default=None,
                    help="probe order: 0 by the learned distinct ratio, 1 claim first, 2 read first")
    ap.add_argument("--item-kmers", type=int, default=None,
                    help="k-mers per insert work item: 64, 128 or 256 (default)")
    ap.add_argument("--load-factor", type=float, default=None, help="table load factor (0.5)")
    ap.add_argument("--ksweep", action="store_true",
                    help="throughput against k from 32 to 479 on one long-read workload")
    ap.add_argument("--ks", default=None, help="comma-separated k values of --ksweep (default all)")
    ap.add_argument("--ksweep-genome", type=int, default=10_000_000,
                    help="genome length of the --ksweep workload (bases)")
    ap.add_argument("--ksweep-windows", type=int, default=400_000,
                    help="k-mer windows of the oracle's sample at every k of --ksweep")
    ap.add_argument("--orderings", action="store_true",
                    help="compare the minimizer orderings (super-mers vs largest bin) instead")
    ap.add_argument("--serving-jobs", type=int, default=48,
                    help="jobs of the serving stream (--workload %s)" % SERVING_WORKLOAD)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-budget-gb", type=float, default=150.0)
    ap.add_argument("--serving-scale", type=float, default=1.0,
                    help="shrink every serving job's genome and reads by this factor")
    ap.add_argument("--serving-rate", type=float, default=20.0, help="mean arrivals per second")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the configs block (the other workloads and the serving stream)")
    ap.add_argument("--config-steps", type=int, default=5,
                    help="timed steps of every workload of the configs block")
    ap.add_argument("--config-sample-windows", type=int, default=300_000,
                    help="k-mer windows of each config's oracle-checked read sample")
    ap.add_argument("--no-serving", action="store_true", help="configs block without serving")
    ap.add_argument("--steps-only", action="store_true",
                    help="only the timed steps of the headline workload (for launch lists): no "
                         "membench, batched-vs-per-bin, probe statistics, App. C, e2e, oracle "
                         "or configs block")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce(x: float, dist, device, op: str) -> float:
    """x reduced over the ranks ("max" or "sum"); x itself on one process."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _replica_value(units_per_rank: int, local_ms: float, dist, world: int, device) -> tuple:
    """Whole-job throughput of independent replicas: the units of all ranks over the slowest
    rank's time.  Returns (units per second, max ms)."""
    ms = _reduce(local_ms, dist, device, "max")
    return units_per_rank * world / (ms / 1000.0), ms


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _src_sha():
    """sha-256 (16 hex digits) of the phase-two kernel sources."""
    h = hashlib.sha256()
    for f in ("count.cu", "insert.cuh", "insert_w1_2.cu", "insert_w3.cu", "insert_w4.cu",
              "insert_w5_7.cu", "insert_w8_11.cu", "insert_w12_15.cu", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_1607_06618_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_and_source(workload: str, kernel: str = "insert_kernel"):
    """(dram bytes per launch of the kernel, where they come from) from the committed ncu
    summary profiles/<kernel>_<workload>.md; (None, why) when there is none or the kernel
    source changed since it was taken."""
    rel = os.path.join("profiles", "%s_%s.md" % (kernel, workload))
    try:
        text = open(os.path.join(ROOT, rel)).read()
    except OSError:
        return None, "no ncu summary for this workload"
    sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    tr = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not sha or not tr:
        return None, "%s holds no traffic line" % rel
    if sha.group(1) != _src_sha():
        return None, "%s was taken on another kernel source" % rel
    return int(tr.group(1)), "%s (ncu dram__bytes_read + write, source %s)" % (rel, sha.group(1))


class Clocks:
    """nvidia-smi sampler running while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _model_bytes(occ, n_bases, distinct, emitted, W):
    """Algorithmic bytes: occ*(b_in + P(W)) for the insert kernel; + distinct*(8W+8) +
    emitted*(8W+4) for the whole phase two."""
    P = 32 * (-(-(8 * W + 8) // 32)) + 32
    b_in_total = 0.25 * n_bases
    insert = b_in_total + occ * P
    step = insert + distinct * (8 * W + 8) + emitted * (8 * W + 4)
    return insert, step


def _reads_for_windows(offs, k, target):
    """Smallest n such that the first n reads hold at least ``target`` k-windows (N ignored)."""
    lens = np.diff(offs.astype(np.int64))
    cum = np.cumsum(np.maximum(lens - k + 1, 0))
    return int(min(offs.size - 1, np.searchsorted(cum, target) + 1))


def run_cpu_oracle(seq, offs, p, windows_sample):
    """The oracle on the first reads holding about ``windows_sample`` k-mer windows."""
    import oracle
    n = _reads_for_windows(offs, p["k"], windows_sample)
    s, o = seq[: int(offs[n])], offs[: n + 1]
    t0 = time.perf_counter()
    keys, counts = oracle.count(s, o, p["k"], canonical=True, min_count=p["min_count"])
    dt = time.perf_counter() - t0
    occ = oracle.windows(s, o, p["k"])
    return occ, dt, n


def _host_workload(name):
    from paper_1607_06618_b300 import synth
    if name in synth.TORCH_WORKLOADS:
        s, o, p = synth.torch_workload(name, device="cpu")
        return s.numpy(), o.numpy().view(np.uint64), p
    return synth.workload(name)


CONFIG_WORKLOADS = ("uniform-20k-k32", "genome100M-repeats-30x-k99", "genome50M-longreads-20x-k200")


def _device_workload(name):
    """(seq uint8, offsets int64) CUDA tensors and the parameters of a named workload."""
    import torch
    from paper_1607_06618_b300 import synth
    if name in synth.TORCH_WORKLOADS:
        return synth.torch_workload(name, device="cuda")
    seq, offs, p = synth.workload(name)
    return torch.from_numpy(seq).cuda(), torch.from_numpy(offs.view(np.int64)).cuda(), p


def _insert_kernel_name(k, opts, fused):
    W = (2 * k + 63) // 64
    WS = 1 if 2 * k <= 93 else (2 * k - 30 + 62) // 63  # stored chunks beyond the 30-bit tag
    return ("fused_kernel<%d,%d>" if fused else "insert_kernel<%d,%d>") % (W, WS)


def _roofline(ph, steps, occ, n_bases, info, k, workload, hbm, peak_kind, opts):
    """Roofline of the dominant kernel (insert, or the fused kernel) from its event-timed
    launches: the byte model per launch / average launch time, against the HBM peak."""
    W = (2 * k + 63) // 64
    insert_bytes, step_bytes = _model_bytes(occ, n_bases, info["distinct"], info["emitted"], W)
    ins_ms = ph["insert_ms"] / max(1, ph["insert_launches"])
    fused = ph["compact_ms"] == 0.0  # fused form: one kernel inserts and compacts
    kbytes = step_bytes if fused else insert_bytes
    achieved = kbytes / (ins_ms / 1000.0) / 1e9
    kname = _insert_kernel_name(k, opts, fused)
    traffic, traffic_from = _traffic_and_source(workload, kname.split("<")[0])
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "traffic_from": traffic_from,
            "kernel": kname,
            "peak_kind": peak_kind + " (hbm_gbs, copy bandwidth)",
            "bytes_per_launch": kbytes, "launch_ms": ins_ms}, step_bytes


def _time_steps(ctx, stream, s_dev, o_dev, p, opts, steps, warmup, dist=None, clocks_dev=None):
    """Warm-up, then ``steps`` event-timed steps (gerbil_partition + gerbil_count_batch over all
    bins) with the context's phase events on, bracketed by a barrier (under torchrun) and a
    device synchronisation on both sides; nvidia-smi samples the clocks meanwhile.  Returns
    (info of a warm-up step, ms per step, phase times summed over the steps, clocks)."""
    import torch
    k, m, nbins, mc = p["k"], p["m"], p["nbins"], p["min_count"]
    bb = p.get("bin_bounds")
    info = {}

    def step(record=False):
        bins = ctx.partition(s_dev, o_dev, k, m, nbins, opts, bb)
        res = ctx.count_batch(bins, None, k, mc, opts)
        st = res.info()[2]
        if record:
            info.update(st)
            info["n_supermers"] = bins.info()["n_supermers"]
        res.free()
        bins.free()
        return st

    nwarm = max(3, warmup)
    for i in range(nwarm):
        step(record=(i == nwarm - 1))
    ctx.profile(True)
    clocks = Clocks(clocks_dev if clocks_dev is not None else torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st = step()
        assert st["emitted"] == info["emitted"] and st["occurrences"] == info["occurrences"]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    ph = ctx.phase_times()
    ctx.profile(False)
    return info, ms / steps, ph, ck


def _batched_vs_per_bin(gerbil, torch, ctx, s_dev, o_dev, p, opts, reps, variants):
    """Phase two over all bins, host-timed per call with a device synchronisation: one
    count_batch per variant (default: the persistent insert grid + compaction grid) against
    one gerbil_count call per bin.  The autotuned variant is tuned by an untimed first call."""
    k, m, nbins, mc = p["k"], p["m"], p["nbins"], p["min_count"]
    bins = ctx.partition(s_dev, o_dev, k, m, nbins, opts, p.get("bin_bounds"))
    torch.cuda.synchronize()

    def host_ms(o):
        ctx.count_batch(bins, None, k, mc, o).free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.count_batch(bins, None, k, mc, o).free()
        torch.cuda.synchronize()
        return 1000 * (time.perf_counter() - t0) / reps

    out = {}
    for name, o in variants:
        t0 = time.perf_counter()
        if name == "batched_autotune_ms":
            out["autotune_s"] = 0.0
            ctx.count_batch(bins, None, k, mc, o).free()  # tunes on first use
            torch.cuda.synchronize()
            out["autotune_s"] = time.perf_counter() - t0
            out["autotune"] = ctx.get_tuning(k)
        out[name] = host_ms(o)
    ctx.count(bins, 0, k, mc, opts).free()
    torch.cuda.synchronize()
    tp = time.perf_counter()
    for _ in range(reps):
        for b in range(nbins):
            ctx.count(bins, b, k, mc, opts).free()
    torch.cuda.synchronize()
    out["per_bin_ms"] = 1000 * (time.perf_counter() - tp) / reps
    out["speedup"] = out["per_bin_ms"] / out["batched_ms"]
    bins.free()
    return out


def _sample_check(gerbil, ctx, s_dev, o_dev, p, opts, windows_sample):
    """The oracle (one core) on the first reads holding about ``windows_sample`` k-mer windows,
    timed, and the same reads counted on the GPU (min_count 1, host buffers): row for row
    equality and the oracle's rate."""
    import oracle
    k = p["k"]
    offs = o_dev.cpu().numpy().view(np.uint64)
    n = _reads_for_windows(offs, k, windows_sample)
    so = offs[: n + 1].copy()
    ss = s_dev[: int(so[-1])].cpu().numpy()
    t0 = time.perf_counter()
    oracle.count(ss, so, k, canonical=True, min_count=p["min_count"])
    dt = time.perf_counter() - t0
    occ_s = oracle.windows(ss, so, k)
    wk, wc = oracle.count(ss, so, k, canonical=True, min_count=1)
    bins = ctx.partition(ss, so, k, p["m"], p["nbins"], opts, p.get("bin_bounds"))
    res = ctx.count_batch(bins, None, k, 1, opts)
    gk, gc = res.to_host()
    res.free()
    bins.free()
    W = (2 * k + 63) // 64
    gk = np.asarray(gk, dtype=np.uint64).reshape(len(gc), W)
    order = np.lexsort(gk.T[::-1]) if len(gc) else np.zeros(0, np.int64)
    same = bool(len(gc) == len(wc)
                and np.array_equal(gk[order], np.asarray(wk, np.uint64).reshape(len(wc), W))
                and np.array_equal(np.asarray(gc, np.uint64)[order], np.asarray(wc, np.uint64)))
    return {"sample_bit_exact": same, "sample_rows": int(len(wc)), "sample_windows": int(occ_s),
            "sample_reads": int(n), "oracle_kmers_per_s": occ_s / dt, "oracle_cores": 1,
            "oracle_s": dt}


def run_config(a, name, local, hbm, peak_kind):
    """One config of the configs block: event-timed steps with the insert kernel's roofline,
    batched vs per-bin phase two, and an oracle-checked read sample."""
    import torch
    from paper_1607_06618_b300 import gerbil
    t_gen = time.perf_counter()
    s_dev, o_dev, p = _device_workload(name)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    k = p["k"]
    stream = torch.cuda.current_stream()
    ctx = gerbil.Context(local, stream=stream.cuda_stream)
    opts = gerbil.default_opts()
    try:
        info, ms, ph, ck = _time_steps(ctx, stream, s_dev, o_dev, p, opts, a.config_steps, 3,
                                       clocks_dev=local)
        occ = info["occurrences"]
        n_bases = occ + info["n_supermers"] * (k - 1)
        roof, step_bytes = _roofline(ph, a.config_steps, occ, n_bases, info, k, name, hbm, peak_kind,
                                     opts)
        variants = [("batched_ms", opts), ("batched_graph_ms", gerbil.default_opts(graph=1))]
        if name == "genome100M-repeats-30x-k99":
            variants.append(("batched_autotune_ms", gerbil.default_opts(autotune=1)))
        bvp = _batched_vs_per_bin(gerbil, torch, ctx, s_dev, o_dev, p, opts, a.per_bin_steps, variants)
        chk = _sample_check(gerbil, ctx, s_dev, o_dev, p, opts, a.config_sample_windows)
    finally:
        ctx.close()
    out = {"value": occ / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms, "steps": a.config_steps,
           "warmup": 3, "config": _config(name, p, s_dev, o_dev), "generation_s": t_gen,
           "occurrences_per_step": occ, "distinct": info["distinct"], "emitted": info["emitted"],
           "supermers": info["n_supermers"], "table_slots": info["table_slots"],
           "overflowed": info["overflowed"], "groups": info["groups"], "roofline": roof,
           "phase_ms": {key[:-3]: ph[key] / a.config_steps for key in ph if key.endswith("_ms")},
           "gpu_launches": int(ph["kernel_launches"]), "batched_vs_per_bin": bvp, "clocks": ck}
    out.update(chk)
    del s_dev, o_dev
    torch.cuda.empty_cache()
    return out



def main_reference(a, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    seq, offs, p = _host_workload(a.workload)
    for _ in range(a.warmup):
        run_cpu_oracle(seq, offs, p, a.ref_sample_windows)
    times, occ = [], 0
    for _ in range(a.steps):
        occ, dt, n = run_cpu_oracle(seq, offs, p, a.ref_sample_windows)
        times.append(dt)
    total = sum(times)
    value = occ * a.steps / total
    sample = "first %d of %d reads per step (%d k-mer windows)" % (n, offs.size - 1, occ)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": _config(a.workload, p, seq, offs),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "nproc": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(name, p, seq, offs):
    nreads = int(offs.numel() if hasattr(offs, "numel") else offs.size) - 1
    nbases = int(seq.numel() if hasattr(seq, "numel") else seq.size)
    return {"workload": name, "k": p["k"], "m": p["m"], "nbins": p["nbins"],
            "bins": "log-normal shares (sigma 1)" if p.get("bin_bounds") is not None else "uniform",
            "min_count": p["min_count"], "reads": nreads,
            "bases": nbases, "mode": "count_batch over all bins (persistent insert grid)",
            "l2": ("inputs larger than L2 (%.0f MB ASCII reads > 126 MB)" % (nbases / 1e6)
                   if nbases > L2_BYTES else
                   "inputs smaller than L2 (%.1f MB); tables and bins rewritten every step"
                   % (nbases / 1e6))}


def main_ours(a, world, rank, local):
    import torch
    from paper_1607_06618_b300 import gerbil, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if a.workload in synth.TORCH_WORKLOADS:  # drawn on the GPU, copied to the host once
        s_dev, o_dev, p = synth.torch_workload(a.workload, device="cuda")
        seq, offs = s_dev.cpu().numpy(), o_dev.cpu().numpy().view(np.uint64)
    else:
        seq, offs, p = synth.workload(a.workload)
        s_dev = torch.from_numpy(seq).cuda()
        o_dev = torch.from_numpy(offs.view(np.int64)).cuda()
    k, m, nbins, mc = p["k"], p["m"], p["nbins"], p["min_count"]
    bb = p.get("bin_bounds")
    W = (2 * k + 63) // 64
    stream = torch.cuda.current_stream()
    ctx = gerbil.Context(local, stream=stream.cuda_stream)
    kw = {}
    if a.fused is not None:
        kw["fused"] = a.fused
    if a.schedule is not None:
        kw["schedule"] = a.schedule
    if a.autotune:
        kw["autotune"] = 1
    if a.graph:
        kw["graph"] = 1
    if a.probe_scheme is not None:
        kw["probe_scheme"] = a.probe_scheme
    if a.item_kmers is not None:
        kw["item_kmers"] = a.item_kmers
    if a.claim_first is not None:
        kw["claim_first"] = a.claim_first
    if a.load_factor is not None:
        kw["load_factor"] = a.load_factor
    opts = gerbil.default_opts(**kw)

    # warm-up steps, then exactly a.steps event-timed steps between device synchronisations
    info, ms1, ph, ck = _time_steps(ctx, stream, s_dev, o_dev, p, opts, a.steps, a.warmup, dist,
                                    local)
    occ = info["occurrences"]
    n_bases = occ + info["n_supermers"] * (k - 1)
    value, ms = _replica_value(occ * a.steps, ms1 * a.steps, dist, world, "cuda")

    # roofline of the dominant kernel (insert), from its own event-timed launches
    hbm, peak_kind = _peaks()
    roofline, step_bytes = _roofline(ph, a.steps, occ, n_bases, info, k, a.workload, hbm, peak_kind,
                                     opts)
    ins_ms = roofline["launch_ms"]
    p2_ms = (ph["clear_ms"] + ph["insert_ms"] + ph["compact_ms"] + ph["overflow_ms"]) / a.steps
    phase_ms = {key[:-3]: ph[key] / a.steps for key in ph if key.endswith("_ms")}

    # ceilings of the operations the insert kernel is made of (random 32-byte slot load, then
    # an atomic add on it), L2-resident and HBM-sized, measured on this GPU
    membench = None
    if rank == 0 and not a.steps_only:
        membench = {}
        for label, nbytes in (("l2_32MB", 32 << 20), ("hbm_4GB", 4 << 30)):
            for op, name in ((0, "red"), (1, "load32"), (2, "load32_then_red"), (3, "cas")):
                membench["%s_%s_gops" % (label, name)] = gerbil.gerbil_membench(ctx.handle, nbytes, op, 256)
        ins_rate = occ / (ins_ms / 1000.0) / 1e9
        roofline["l2_ops"] = {
            "achieved": ins_rate, "unit": "G inserts/s",
            "peak": membench["l2_32MB_load32_then_red_gops"],
            "frac": ins_rate / membench["l2_32MB_load32_then_red_gops"],
            "peak_kind": "measured in this run: random 32-byte slot load then atomic add, "
                         "32 MB footprint (gerbil_membench op 2)"}

    # batched (one persistent launch) vs one count call per bin, phase two only
    bvp = None
    if a.per_bin_steps > 0 and rank == 0 and not a.steps_only:
        variants = [("batched_ms", opts), ("batched_fused_ms", gerbil.default_opts(fused=1)),
                    ("batched_static_schedule_ms", gerbil.default_opts(schedule=0)),
                    ("batched_waves_ms", gerbil.default_opts(fused=2)),
                    ("batched_graph_ms", gerbil.default_opts(graph=1)),
                    ("batched_autotune_ms", gerbil.default_opts(autotune=1))]
        bvp = _batched_vs_per_bin(gerbil, torch, ctx, s_dev, o_dev, p, opts, a.per_bin_steps, variants)
        bvp["what"] = ("phase two over all %d bins, host-timed: one count_batch per variant "
                       "(default: persistent insert grid + compaction grid; fused queue kernel; "
                       "static schedule; waves; CUDA graph; autotuned) against %d count calls"
                       % (nbins, nbins))

    # probe statistics of one step's phase two under both probe schemes, on the same bins and
    # table sizes (Sec. 3.3 compares one-by-one probing, 90.37% at the first probe and at most
    # 29, with 128-byte window probing, 99.94% and at most 7): share placed at the first slot
    # read / within the first line or window, the most slots / lines any k-mer needed, and the
    # phase-two time of each scheme; recorded outside the timed region
    probes = None
    if rank == 0 and not a.steps_only:
        bins = ctx.partition(s_dev, o_dev, k, m, nbins, opts, bb)

        def _maxb(h):
            nz = [i for i in range(33) if h[i]]
            return (nz[-1] + 1) if nz else 0

        probes = {}
        for name, scheme in (("linear", 0), ("windowed", 1)):
            o = gerbil.default_opts(**dict(kw, probe_scheme=scheme))
            ctx.probe_stats(True)
            ctx.count_batch(bins, None, k, mc, o).free()
            hs_, hl_ = ctx.get_probe_stats()
            ctx.probe_stats(False)
            tot = float(hs_.sum())
            ctx.profile(True)
            for _ in range(3):
                ctx.count_batch(bins, None, k, mc, o).free()
            php = ctx.phase_times()
            ctx.profile(False)
            probes[name] = {
                "first_slot_share": float(hs_[0]) / tot, "first_line_share": float(hl_[0]) / tot,
                "max_slots": _maxb(hs_), "max_lines": _maxb(hl_),
                "mean_slots": float(sum((i + 1) * int(hs_[i]) for i in range(33))) / tot,
                "mean_lines": float(sum((i + 1) * int(hl_[i]) for i in range(33))) / tot,
                "overflowed": int(hs_[33]),
                "insert_ms": php["insert_ms"] / 3, "phase2_ms": (php["clear_ms"] + php["insert_ms"] +
                                                                php["compact_ms"] + php["overflow_ms"]) / 3}
        probes["what"] = ("per inserted k-mer: slots read until placed and 128-byte lines (linear "
                          "probing) or windows (windowed double hashing) among them; a bucket "
                          "of 33 means 33 or more")
        bins.free()

    # App. C output records of one step's result, written on the device (event-timed)
    appc = None
    if rank == 0 and not a.steps_only:
        bins = ctx.partition(s_dev, o_dev, k, m, nbins, opts, bb)
        res = ctx.count_batch(bins, None, k, mc, opts)
        res.encode_records(k, device=True)  # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        buf = res.encode_records(k, device=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ems = ev0.elapsed_time(ev1)
        appc = {"rows": len(res), "bytes": int(buf.numel()), "ms": ems,
                "what": "size pass + record pass (gerbil_encode_records, device output), "
                        "including its host synchronisation"}
        del buf
        res.free()
        bins.free()

    # end to end through the public API from pinned host buffers, result read back to host:
    # every step copies its reads in, partitions, counts and reads its rows back.  With
    # --e2e-workers W > 1, W host threads each drive a context of their own (own CUDA stream
    # and pinned buffers), so one step's copies overlap another step's kernels.
    e2e = None
    if a.e2e_steps > 0 and not a.steps_only:
        import threading
        nrow = info["emitted"]
        nw = max(1, a.e2e_workers)
        # every worker holds tables of its own: no more workers than sets of tables fit in half
        # the device (one for the 126 GB tables of the long-read workload)
        slot_bytes = gerbil.slot_bytes(k)
        half = torch.cuda.get_device_properties(local).total_memory // 2
        nw = max(1, min(nw, half // max(1, info["table_slots"] * slot_bytes)))
        seq_pin = torch.from_numpy(seq).pin_memory()
        offs_pin = torch.from_numpy(offs.view(np.int64)).pin_memory()
        hs, ho = seq_pin.numpy(), offs_pin.numpy().view(np.uint64)
        workers, wstreams = [], []
        for wid in range(nw):
            if nw == 1:
                wctx = ctx
            else:  # a non-blocking stream each (the legacy default stream would serialise them)
                wstreams.append(torch.cuda.Stream(local))
                wctx = gerbil.Context(local, stream=wstreams[-1].cuda_stream)
            keys_pin = torch.empty((max(1, nrow), W), dtype=torch.int64).pin_memory()
            cnt_pin = torch.empty(max(1, nrow), dtype=torch.int32).pin_memory()
            workers.append((wctx, keys_pin, cnt_pin))

        # the result a step hands back: App. C records (the counter's output format: 1 or 5
        # bytes of count, then 4 bases per byte), or the rows (key words + 32-bit count)
        rec_bytes = []
        for wctx, _, _ in workers:
            bins = wctx.partition(hs, ho, k, m, nbins, opts, bb)
            res = wctx.count_batch(bins, None, k, mc, opts)
            rec_bytes.append(int(gerbil.gerbil_encode_records(res.handle, k)))
            res.free()
            bins.free()
        # room for every count in its 5-byte form: the encoder then skips its size pass
        rec_room = max(1, nrow * ((k + 3) // 4 + 5), rec_bytes[0])
        rec_pin = [torch.empty(rec_room, dtype=torch.uint8).pin_memory() for _ in workers]

        def e2e_step(i, result):
            wctx, kp, cp = workers[i]
            bins = wctx.partition(hs, ho, k, m, nbins, opts, bb)
            res = wctx.count_batch(bins, None, k, mc, opts)
            if result == "records":
                gerbil.gerbil_encode_records(res.handle, k, rec_pin[i].data_ptr(), rec_pin[i].numel(), 0)
            else:
                gerbil.gerbil_counts_to_host(res.handle, kp.numpy().view(np.uint64),
                                             cp.numpy().view(np.uint32))
            res.free()
            bins.free()

        def threaded(share, result):
            errors = []

            def run(i):
                try:
                    for _ in range(share[i]):
                        e2e_step(i, result)
                except Exception as exc:  # reported after the join
                    errors.append(exc)

            threads = [threading.Thread(target=run, args=(i,)) for i in range(nw)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            if errors:
                raise errors[0]

        def run_e2e(result):
            # warm-up: every worker once alone (ratio learning, scratch growth), then two steps
            # each with all workers at once, so that the memory pool has grown to what the
            # concurrent steps hold before the clock starts
            for i in range(nw):
                e2e_step(i, result)
            threaded([2] * nw, result)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            share = [a.e2e_steps // nw + (1 if i < a.e2e_steps % nw else 0) for i in range(nw)]
            runs = []
            for _ in range(3):  # the median of three timed runs (the host threads' timing varies)
                t0 = time.perf_counter()
                threaded(share, result)
                torch.cuda.synchronize()
                runs.append((time.perf_counter() - t0) / a.e2e_steps)
            te = statistics.median(runs)
            val, te_ms = _replica_value(occ, 1000 * te, dist, world, "cuda")
            d2h = rec_bytes[0] if result == "records" else int(nrow * (8 * W + 4))
            return {"value": val, "unit": UNIT, "h2d_bytes_per_step": int(seq.nbytes + offs.nbytes),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": te_ms,
                    "workers": nw, "steps": a.e2e_steps, "result": result,
                    "runs_ms_per_step": [1000 * r for r in runs],
                    "what": "host wall clock over all steps (median of three runs); each step: reads "
                            "copied from pinned host memory, gerbil_partition + gerbil_count_batch, "
                            "then %s copied to pinned host memory; %d host threads with a context "
                            "(stream) each"
                            % ("the App. C output records (gerbil_encode_records)" if result == "records"
                               else "the rows (gerbil_counts_to_host)", nw)}

        # the step's result is the counter's output, App. C records; the rows (key words and a
        # 32-bit count, 55% more bytes back) are measured beside it
        e2e = run_e2e("records")
        e2e_rows = run_e2e("rows")
        for wctx, _, _ in workers:
            if wctx is not ctx:
                wctx.close()
        e2e["rows_instead"] = {key: e2e_rows[key] for key in
                               ("value", "d2h_bytes_per_step", "ms_per_step", "runs_ms_per_step")}

    # the oracle on one core over a bounded sample (cpu_baseline), and the same reads counted
    # on the GPU: row-for-row equality
    cpu = None
    if rank == 0 and not a.no_cpu_baseline and not a.steps_only:
        chk = _sample_check(gerbil, ctx, s_dev, o_dev, p, opts, a.cpu_sample_windows)
        cpu = {"value": chk["oracle_kmers_per_s"], "unit": UNIT, "cores": 1,
               "nproc": os.cpu_count(), "kind": "oracle",
               "sample": "first %d of %d reads (%d k-mer windows), std::map oracle, %.1f s"
                         % (chk["sample_reads"], offs.size - 1, chk["sample_windows"], chk["oracle_s"]),
               "sample_bit_exact": chk["sample_bit_exact"], "sample_rows": chk["sample_rows"]}
    tuning = ctx.get_tuning(k) if (a.autotune or bvp) else None
    ctx.close()
    del s_dev, o_dev
    torch.cuda.empty_cache()

    # the other workloads (configs 1, 3, 4) and the serving stream, each measured on its own
    configs = None
    if rank == 0 and not a.no_configs and not a.steps_only:
        configs = {}
        for name in CONFIG_WORKLOADS:
            configs[name] = run_config(a, name, local, hbm, peak_kind)
        if not a.no_serving:
            configs[SERVING_WORKLOAD] = run_serving(a, local, None, 3)
        rows, ck_k, _, _, G = _ksweep(a, local, KSWEEP_CONFIG_KS, a.config_steps, 3)
        configs["ksweep-genome%gM-1000bp-20x" % (G / 1e6)] = {
            "workload": "genome%gM-1000bp-20x, 0.2%% substitutions, m=11, 512 bins, min count 2"
                        % (G / 1e6), "what": "keys of 10 to 15 words (k = 320, 400, 479)",
            "clocks": ck_k, "results": rows}

    if rank == 0:
        cfg = _config(a.workload, p, seq, offs)
        cfg.update({"occurrences_per_step": occ, "distinct": info["distinct"],
                    "emitted": info["emitted"], "supermers": info["n_supermers"],
                    "table_slots": info["table_slots"], "overflowed": info["overflowed"]})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": cfg, "roofline": roofline,
            "step_model": {"bytes": step_bytes, "phase2_ms": p2_ms,
                           "achieved_gbs": step_bytes / (p2_ms / 1000.0) / 1e9},
            "phase_ms": phase_ms, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck,
            "gpu_launches": int(ph["kernel_launches"]), "batched_vs_per_bin": bvp,
            "appc_records": appc, "probe_stats": probes,
            "opts": {key: val for key, val in kw.items()},
            "autotune": tuning,
            "membench": membench,
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[i]


def run_serving(a, local, dist=None, warmup=3):
    """Counting jobs arriving as a Poisson stream, served by gerbil.Server under an HBM budget:
    aggregate k-mers/s over the whole stream (first arrival to last result) and the p50/p99
    of the job latency (arrival to result on the device), host wall clock.  Every job's reads
    are drawn on the device before the clock starts; results stay on the device and are freed
    once waited for.  Each rank serves its own stream (replicas).  Returns a dict."""
    import threading
    import torch
    from paper_1607_06618_b300 import gerbil, synth

    t_gen = time.perf_counter()
    jobs = synth.serving_jobs(a.serving_jobs, rate=a.serving_rate)
    reads = [synth.t_serving_reads(j, "cuda", a.serving_scale) for j in jobs]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    budget = int(a.serving_budget_gb * 1e9)

    def run_stream(server, order, arrivals):
        ids = [None] * len(order)
        t0 = time.perf_counter()

        def submitter():
            for x, j in enumerate(order):
                delay = t0 + arrivals[x] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                jb = jobs[j]
                s, o = reads[j]
                ids[x] = server.submit(s, o, jb["k"], jb["m"], jb["nbins"], jb["min_count"])

        th = threading.Thread(target=submitter)
        th.start()
        out = []
        for x in range(len(order)):
            while ids[x] is None:
                time.sleep(0.0005)
            res, times = server.wait(ids[x])
            n, W, st = res.info()
            res.free()
            out.append(dict(times, occurrences=st["occurrences"], rows=n, groups=st["groups"]))
        th.join()
        return time.perf_counter() - t0, out

    # warm-up: the smallest jobs, all at once
    server = gerbil.Server(local, budget, a.serving_slots)
    small = sorted(range(len(jobs)), key=lambda j: jobs[j]["nreads"])[:max(3, warmup)]
    run_stream(server, small, [0.0] * len(small))
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    wall, out = run_stream(server, list(range(len(jobs))), [j["arrival_s"] for j in jobs])
    ck = clocks.stop()
    st = server.stats()
    server.close()
    bases = int(sum(int(r[0].numel()) for r in reads))
    del reads
    torch.cuda.empty_cache()
    occ = sum(r["occurrences"] for r in out)
    lat = [r["latency_ms"] for r in out]
    return {
        "workload": SERVING_WORKLOAD, "value": occ / wall, "unit": UNIT, "jobs": len(jobs),
        "warmup_jobs": len(small), "rate_jobs_per_s": a.serving_rate, "slots": a.serving_slots,
        "hbm_budget_bytes": budget, "scale": a.serving_scale, "bases_total": bases,
        "occurrences_total": occ,
        "k_mix": {str(k): sum(1 for j in jobs if j["k"] == k) for k, _ in synth.SERVING_K},
        "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "mean": statistics.mean(lat),
                       "max": max(lat)},
        "queue_ms": {"p50": _pct([r["queue_ms"] for r in out], 50),
                     "p99": _pct([r["queue_ms"] for r in out], 99)},
        "run_ms": {"p50": _pct([r["run_ms"] for r in out], 50),
                   "p99": _pct([r["run_ms"] for r in out], 99)},
        "makespan_s": wall, "last_arrival_s": jobs[-1]["arrival_s"],
        "offered_kmers_per_s": occ / max(1e-9, jobs[-1]["arrival_s"]),
        "saturated": wall > 1.1 * jobs[-1]["arrival_s"],
        "server": st, "jobs_grouped": sum(1 for r in out if r["groups"] > 1), "clocks": ck,
        "generation_s": t_gen,
        "timing": "host wall clock from the first arrival to the last result; device-resident reads",
    }


def main_serving(a, world, rank, local):
    """The serving stream alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = run_serving(a, local, dist, a.warmup)
    value = _reduce(r["value"], dist, "cuda", "sum")
    if rank == 0:
        line = {
            "metric": "serving: aggregate canonical k-mers counted/sec, p50/p99 job latency",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": r["jobs"],
            "warmup": r["warmup_jobs"], "ms_per_step": 1000 * r["makespan_s"] / r["jobs"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {key: r[key] for key in ("workload", "jobs", "rate_jobs_per_s", "slots",
                                               "hbm_budget_bytes", "scale", "bases_total",
                                               "occurrences_total", "k_mix")},
            "clocks": r["clocks"], "gpu_launches": int(r["server"]["kernel_launches"]),
            "cpu_baseline": None, "e2e": None,
        }
        line.update({key: r[key] for key in ("latency_ms", "queue_ms", "run_ms", "makespan_s",
                                             "last_arrival_s", "offered_kmers_per_s", "saturated",
                                             "server", "jobs_grouped", "timing")})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main_orderings(a, rank, local):
    """Sec. 3.1's trade-off between the orderings, on the GPU partition of a synthetic read set:
    super-mers and their packed bytes (the paper's temporary-file size) against the largest
    k-mer count of one minimizer (with 65,536 bins, about one minimizer per bin for m = 6)."""
    import torch
    from paper_1607_06618_b300 import gerbil, synth
    torch.cuda.set_device(local)
    seq, offs, p = synth.workload(a.workload)
    s_dev = torch.from_numpy(seq).cuda()
    o_dev = torch.from_numpy(offs.view(np.int64)).cuda()
    ctx = gerbil.Context(local)
    variants = [("kmc2", 0, 0.5), ("lex", 1, 0.5), ("cgat", 2, 0.5), ("roberts", 3, 0.5),
                ("random", 4, 0.5), ("dfp0", 5, 0.0), ("dfp0.5", 5, 0.5), ("dfp0.8", 5, 0.8),
                ("dfp1", 5, 1.0)]
    out = {}
    for k, m in ((28, 6), (p["k"], p["m"])):
        nb = 65536
        for name, o, piv in variants:
            bins = ctx.partition(s_dev, o_dev, k, m, nb,
                                 gerbil.default_opts(ordering=o, dfp_pivot=piv))
            inf = bins.info()
            per = [gerbil.gerbil_bin_stats(bins.handle, b) for b in range(nb)]  # (super, bases, k-mers)
            kmers = np.array([x[2] for x in per], dtype=np.float64)
            nbases = sum(x[1] for x in per)
            bins.free()
            out["k%d_m%d_%s" % (k, m, name)] = {
                "supermers": int(inf["n_supermers"]), "packed_bytes": int(nbases // 4),
                "max_kmers_per_bin": int(kmers.max()), "mean_kmers_per_nonempty_bin":
                float(kmers[kmers > 0].mean()), "nonempty_bins": int((kmers > 0).sum())}
    ctx.close()
    if rank == 0:
        print(json.dumps({"experiment": "minimizer orderings (Sec. 3.1, Fig. 3)",
                          "workload": a.workload, "bins": 65536, "results": out}), flush=True)
    return 0


KSWEEP = (32, 48, 65, 99, 127, 150, 200, 256, 320, 400, 479)


KSWEEP_CONFIG_KS = (320, 400, 479)  # the wide-key points carried by the default bench line


def _ksweep(a, local, ks, steps, warmup):
    """Throughput against k on one long-read workload: a 10 Mbp uniform genome (seed 6001;
    --ksweep-genome changes its length), 20x of 1000 bp reads from both strands with 0.2%
    substitutions (seed 6002), m = 11, 512 bins, min count 2.  Per k: the whole step on the GPU
    (event-timed, phase split), the insert kernel's byte model and HBM fraction, and the oracle
    on one core over a bounded sample, whose reads the GPU also counts for a bit-exact check.
    Returns (rows, clocks, HBM peak, peak kind, genome length)."""
    import torch
    import oracle
    from paper_1607_06618_b300 import gerbil, synth
    torch.cuda.set_device(local)
    G, L = a.ksweep_genome, 1000
    gen = synth.t_genome(G, 6001, "cuda")
    s_dev, o_dev = synth.t_sampled_reads(gen, 20 * G // L, L, 0.002, 6002)
    del gen
    seq, offs = s_dev.cpu().numpy(), o_dev.cpu().numpy().view(np.uint64)
    m, nbins, mc = 11, 512, 2
    stream = torch.cuda.current_stream()
    ctx = gerbil.Context(local, stream=stream.cuda_stream)
    opts = gerbil.default_opts(**({} if a.claim_first is None else {"claim_first": a.claim_first}))
    hbm, peak_kind = _peaks()
    rows = []
    clocks = Clocks(local)
    for k in ks:
        W = (2 * k + 63) // 64
        info = {}

        def step(record=False):
            bins = ctx.partition(s_dev, o_dev, k, m, nbins, opts)
            res = ctx.count_batch(bins, None, k, mc, opts)
            if record:
                info.update(res.info()[2])
                info["n_supermers"] = bins.info()["n_supermers"]
            res.free()
            bins.free()

        for i in range(max(3, warmup)):
            step(record=(i == 0))
        occ = info["occurrences"]
        n_bases = occ + info["n_supermers"] * (k - 1)
        ctx.profile(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ph = ctx.phase_times()
        ctx.profile(False)
        ins_ms = ph["insert_ms"] / max(1, ph["insert_launches"])
        insert_bytes, _ = _model_bytes(occ, n_bases, info["distinct"], info["emitted"], W)

        # the oracle on the first reads holding about --ksweep-windows windows (timed at the
        # workload's min count); the GPU counts the same reads and must agree row for row with
        # every k-mer of them (min count 1: the sample is too thin for repeats)
        n = _reads_for_windows(offs, k, a.ksweep_windows)
        ss, so = seq[: int(offs[n])], offs[: n + 1]
        t0 = time.perf_counter()
        oracle.count(ss, so, k, canonical=True, min_count=mc)
        dt = time.perf_counter() - t0
        occ_s = oracle.windows(ss, so, k)
        wk, wc = oracle.count(ss, so, k, canonical=True, min_count=1)
        bins = ctx.partition(ss, so, k, m, nbins, opts)
        res = ctx.count_batch(bins, None, k, 1, opts)
        gk, gc = res.to_host()
        res.free()
        bins.free()
        gk = np.asarray(gk, dtype=np.uint64).reshape(len(gc), W)
        order = np.lexsort(gk.T[::-1]) if len(gc) else np.zeros(0, np.int64)
        same = (len(gc) == len(wc)
                and np.array_equal(gk[order], np.asarray(wk, np.uint64).reshape(len(wc), W))
                and np.array_equal(np.asarray(gc, np.uint64)[order], np.asarray(wc, np.uint64)))
        if not same:
            raise SystemExit("k=%d: GPU result differs from the oracle on the sample" % k)
        slot = gerbil.slot_bytes(k)
        rows.append({
            "k": k, "W": W, "slot_bytes": slot, "slots_per_128B_line": round(128 / slot, 3),
            "occurrences": occ, "distinct": info["distinct"], "emitted": info["emitted"],
            "gpu_kmers_per_s": occ / (ms / 1000.0), "ms_per_step": ms,
            "phase_ms": {key[:-3]: ph[key] / steps for key in
                         ("encode_ms", "supermer_ms", "clear_ms", "insert_ms", "compact_ms",
                          "overflow_ms") if key in ph},
            "insert_bytes_per_occ": insert_bytes / occ,
            "insert_hbm_frac": insert_bytes / (ins_ms / 1000.0) / 1e9 / hbm,
            "oracle_kmers_per_s": occ_s / dt, "oracle_sample_windows": occ_s,
            "gpu_over_oracle": (occ / (ms / 1000.0)) / (occ_s / dt), "sample_bit_exact": same,
            "sample_rows_checked": len(wc)})
        torch.cuda.empty_cache()
    ck = clocks.stop()
    ctx.close()
    del s_dev, o_dev
    torch.cuda.empty_cache()
    return rows, ck, hbm, peak_kind, G


def main_ksweep(a, rank, local):
    """Throughput against k (Sec. 4 finds the GPU speed-up of the paper's hybrid counter gone
    beyond k = 150, because fewer wider table entries fit in the parallel window scan), over
    every k of the sweep (or --ks)."""
    ks = tuple(int(x) for x in a.ks.split(",")) if a.ks else KSWEEP
    rows, ck, hbm, peak_kind, G = _ksweep(a, local, ks, a.steps, a.warmup)
    if rank == 0:
        print(json.dumps({"experiment": "throughput against k (Sec. 4, GPU speed-up beyond k = 150)",
                          "workload": "genome%gM-1000bp-20x, 0.2%% substitutions, m=11, 512 "
                                      "bins, min count 2" % (G / 1e6), "steps": a.steps,
                          "hbm_peak_gbs": hbm,
                          "peak_kind": peak_kind, "oracle_cores": 1, "clocks": ck,
                          "results": rows}), flush=True)
    return 0


def main():
    a = _args()
    world, rank, local = _dist()
    if a.orderings:
        return main_orderings(a, rank, local)
    if a.ksweep:
        return main_ksweep(a, rank, local)
    if a.workload == SERVING_WORKLOAD:
        if a.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle counts one input at a time; no serving arm"}))
            return 0
        return main_serving(a, world, rank, local)
    if a.impl == "reference":
        return main_reference(a, world, rank)
    return main_ours(a, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())

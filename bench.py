#!/usr/bin/env python
"""Benchmark of the Digital Brain hot path on one GB300 (or N replicas).

Headline workload (the default): the largest network one GPU holds --
20,000,000 conductance LIF neurons in 200 regions of 100,000 (80 % E /
20 % I), in-degree 1,000 (800 within the region, 200 from excitatory neurons
of other regions drawn from a seeded 200x200 region matrix of density 0.3),
2e10 synapses as 6-byte (target, BF16 weight) records (120 GB), delays
0.1-5 ms within and 5-20 ms across regions, dt = 0.1 ms, drive tuned to
~7 / 15 / 30 Hz (--rate).  Synthetic, seeded; the host graph (140 GB) is
ingested from pageable memory.  One benchmark step = one biological second
(10,000 Euler steps: update, compaction, delivery, region counts, BOLD).

Metric: synaptic events per second (events applied to the accumulators,
counted on the device).  Also reported: real-time factor (wall s per
biological s), neuron updates/s, per-kernel roofline against the measured
HBM copy bandwidth, the end-to-end figure through the C ABI from host
buffers, the CPU oracle timed on the host cores, and compact lines for the
mid-size network, the 10,000-neuron network, the batched HMDA ensemble and
the request server (--no-extras skips them).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--rate 7|15|30]
  python bench.py --workload mid|small|ensemble|serving|nest|columns|dt-study
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
For N > 1, launch with torch.distributed.run; each rank runs an independent
replica (the path does not shard: replicas only) and rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STEPS_PER_BIO_S = 10_000  # dt = 0.1 ms
# Constant current that puts the in-degree-1000 network at the target rate,
# found with paper_2211_15963_gb300.tune.tune_drive on a 1/20 sub-network
# (5 regions of 20,000): 6.9, 14.7 and 29.4 Hz there.
RATE_DRIVE = {7: 3.1757, 15: 7.2221, 30: 16.4246}
UPDATE_BYTES_PER_NEURON = 58   # V r/w 8, J r/w 32, ref r/w 2, accumulator read + clear 16
DELIVER_BYTES_PER_EVENT = 14   # target 4 + BF16 weight 2 + int32 read-modify-write 8
# with two weights per edge: four accumulator channels (read + clear 32) and
# 8-byte records (target 4 + two BF16 weights 4) with an int64 read-modify-write 16
UPDATE_BYTES_PER_NEURON_FOUR = 74
DELIVER_BYTES_PER_EVENT_TWO = 24
METRIC = "synaptic events/s"
UNIT = "events/s"
# (regions, neurons per region) of the two network workloads
WORKLOAD_DIMS = {"large": (200, 100_000), "mid": (100, 20_000)}
# kernels launched per dbnet_step(10,000): 156 replays of the 64-step graph
# (128 launches each; 192 on the pipelined schedule, whose steps are three
# launches, plus the long part launched ahead of the first replay) + 16
# direct steps (2 each) + the graph's base word + the bin close at the end of
# the call; on the persistent schedule one launch per 4,096 steps + the bin
# close
LAUNCHES_PER_BIO_S = 156 * 128 + 16 * 2 + 2
SCHEDULES = {1: "sequential", 2: "pipelined", 3: "persistent"}


def launches_per_call(n_steps, schedule):
    if schedule == "persistent":
        return -(-n_steps // 4096) + 1
    pipelined = schedule == "pipelined"
    chunks, rest = divmod(n_steps, 64)
    return chunks * (192 if pipelined else 128) + 2 * rest + (2 if chunks else 1) + (
        1 if pipelined and chunks else 0)


def parse():
    return parse_from(None)


def parse_from(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--rate", type=int, default=15, choices=sorted(RATE_DRIVE))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--tune-at", type=int, default=2000,
                    help="Euler step at which the library tunes the delivery's launch shape")
    ap.add_argument("--deliver-blocks", type=int, default=0,
                    help="fix the delivery grid (0: automatic; profiling at a chosen grid)")
    ap.add_argument("--step-ms", type=float, default=1000.0,
                    help="biological time per benchmark step of the network workloads (ms); "
                         "shorter steps only for profiling runs")
    ap.add_argument("--profile-steps", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact mid/small/batched/served lines of the default run")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="threads of the oracle's timing variant (0 = every core)")
    ap.add_argument("--regions", type=int, default=None, help="regions of --region-size neurons")
    ap.add_argument("--region-size", type=int, default=None, help="neurons per region")
    ap.add_argument("--pageable", action="store_true",
                    help="host graph in pageable memory (always so for the large workload)")
    ap.add_argument("--k-in", type=int, default=1000, help="in-degree (80 %% within region)")
    ap.add_argument("--two-weights", action="store_true",
                    help="a second weight per edge (four accumulator channels)")
    ap.add_argument("--bin-spikes", action="store_true",
                    help="hand spikes on at the 1 ms bin edges (Supplementary Sec. 3)")
    ap.add_argument("--workload", default="large",
                    choices=["large", "mid", "ensemble", "serving", "nest", "columns", "dt-study",
                             "small"],
                    help="large: the headline line (20 M neurons); mid: 2 M neurons; ensemble: "
                         "64-member HMDA ensemble (steps = TRs) against one network per launch; "
                         "serving: request stream")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--separate-trs", type=int, default=1,
                    help="TRs timed for the one-network-per-launch comparison")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--arrival-hz", type=float, default=4.0)
    ap.add_argument("--catalogue", type=int, default=16,
                    help="distinct request networks built before the stream starts")
    ap.add_argument("--separate-requests", type=int, default=40)
    return ap.parse_args(argv)


def workload_dims(args):
    """(regions, neurons per region) of a network workload."""
    R, S = WORKLOAD_DIMS.get(args.workload, WORKLOAD_DIMS["mid"])
    return (args.regions or R), (args.region_size or S)


def network_name(n):
    return ("largest single-GPU network" if n >= 20_000_000 else
            "mid-size network" if n >= 1_000_000 else "network")


def workload_config(args, rank_count, dims=None):
    two = getattr(args, "two_weights", False)
    R, rs = dims or workload_dims(args)
    n = R * rs
    return {"workload": "%s: %s neurons, %d regions x %s, in-degree %s, dt 0.1 ms, ~%d Hz%s%s"
                        % (network_name(n), f"{n:,}", R, f"{rs:,}", f"{args.k_in:,}", args.rate,
                           ", two weights per edge" if two else "",
                           ", spikes handed on at 1 ms bin edges" if getattr(args, "bin_spikes", False) else ""),
            "weights_per_edge": 2 if two else 1,
            "neurons": n, "regions": R, "in_degree": args.k_in, "synapses": n * args.k_in,
            "dt_ms": 0.1, "target_rate_hz": args.rate, "step": "1 biological second",
            "replicas": rank_count,
            "l2": "flushed (256 MiB write) between timed steps; edge arrays exceed L2"}


def params_for(rate, k_in=1000):
    import synth
    p = synth.scale_for_degree(synth.default_region_params(), k_in)
    p["I_ext"] = RATE_DRIVE[rate]
    return p


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- helpers ----
def rank_seed(rank, large=False):
    """Graph seed of replica `rank` (each rank simulates its own network):
    the largest network's recipe index 4, the mid-size network's 1."""
    import synth
    return synth.seed_for(4 if large else 1) + 1000 * rank


def combine_ranks(events, spikes, neurons, dev_ms, world, device):
    """Whole-job totals over the replicas: events, spikes and neurons summed,
    device time the maximum over ranks (the slowest replica bounds the job)."""
    import torch
    import torch.distributed as dist
    tot = torch.tensor([events, spikes, neurons], dtype=torch.float64, device=device)
    mx = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    e, s, n = (float(x) for x in tot.tolist())
    return e, s, n, float(mx.item())


def kernels_sha():
    p = os.path.join(ROOT, "paper_2211_15963_gb300", "csrc", "kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def measured_traffic(kernel, summary="traffic_mid_network_15hz.md"):
    """DRAM bytes per launch of `kernel` (ncu dram__bytes_read.sum +
    dram__bytes_write.sum) from a committed summary under profiles/ (the
    mid-size network's by default), when it was taken on the current kernel
    source: its line `kernels.cu sha256[:16]: <sha>` must match, and its
    table rows read `| <kernel> | <bytes per launch> | ...`."""
    import re
    p = os.path.join(ROOT, "profiles", summary)
    try:
        txt = open(p).read()
    except OSError:
        return None
    m = re.search(r"kernels\.cu sha256\[:16\]: ([0-9a-f]+)", txt)
    if not m or m.group(1) != kernels_sha():
        return None
    m = re.search(r"^\| %s \| ([0-9]+) \|" % re.escape(kernel), txt, flags=re.M)
    return int(m.group(1)) if m else None


def profiled_shape():
    """Occupancy and issue figures of both kernels from the committed ncu
    full sets (profiles/k_deliver_400k_grid608.md, k_update_400k.md), when
    they were taken on the current kernel source, else None."""
    import re
    out = {}
    for kernel, name, what in (("k_deliver", "k_deliver_400k_grid608.md", "608 blocks"),
                               ("k_update", "k_update_400k.md", "391 tiles")):
        try:
            txt = open(os.path.join(ROOT, "profiles", name)).read()
        except OSError:
            return None
        m = re.search(r"kernels\.cu sha256\[:16\]\s+([0-9a-f]+)", txt)
        if not m or m.group(1) != kernels_sha():
            return None
        warps = re.search(r"^\| warps active[^|]*\| ([0-9.]+) %", txt, flags=re.M)
        issue = re.search(r"^\| issue active \| ([0-9.]+) %", txt, flags=re.M)
        if not warps or not issue:
            return None
        out[kernel] = {"warps_active_pct": float(warps.group(1)), "issue_active_pct": float(issue.group(1)),
                       "source": "profiles/%s (ncu full set, 400,000 neurons, %s)" % (name, what)}
    return out


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def pinned_alloc(torch):
    import numpy as np
    keep = []

    def alloc(n, dt):
        t = torch.empty(n, dtype={np.int32: torch.int32, np.uint16: torch.int16,
                                  np.uint8: torch.uint8}[dt], pin_memory=True)
        keep.append(t)
        return t
    return alloc, keep


def oracle_sample(args, dims, seconds=15.0, onset_steps=500):
    """The CPU oracle (matched FP32) on a bounded sample of a network
    workload, on the host cores: a 1/20-scale network of the same region
    size, in-degree and drive (a twentieth of the regions), run untimed
    past the onset, then timed in 1 ms chunks for about `seconds` of wall
    time.  The oracle runs its all-core timing variant (results identical to
    the single-threaded loop) with --cpu-threads threads (0 = every core)."""
    import oracle
    import synth
    R, S = dims
    r_s = max(1, R // 20)
    g = synth.make_graph([S] * r_s, args.k_in, synth.seed_for(1) + 100,
                         k_within=int(round(0.8 * args.k_in)) if r_s > 1 else args.k_in,
                         d_within=(1, 50), d_cross=(50, 200))
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    s = oracle.Sim(g, params_for(args.rate, args.k_in), seed=synth.seed_for(1) + 1, precision=32,
                   threads=threads)
    s.step(onset_steps)
    i0 = s.info()
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        s.step(10)
        steps += 10
    wall = time.perf_counter() - t0
    i1 = s.info()
    ev = i1["events"] - i0["events"]
    return {"value": ev / wall, "unit": UNIT, "cores": threads, "kind": "oracle",
            "neuron_updates_per_s": g.n_neurons * steps / wall,
            "rtf_of_sample": wall / (steps * 1e-4),
            "cpu": cpu_model(),
            "sample": "%d Euler steps (%.0f ms biological) of a %s-neuron 1/20-scale network "
                      "(%d regions x %s, in-degree %s, same drive) after %d untimed steps; the "
                      "matched-FP32 oracle's all-core timing variant on %d threads"
                      % (steps, steps * 0.1, f"{g.n_neurons:,}", r_s, f"{S:,}", f"{args.k_in:,}",
                         onset_steps, threads)}


def oracle_full_mid(args, onset_steps=500, timed_steps=1000):
    """The CPU oracle (matched FP32, all-core timing variant) on the full
    mid-size network -- the same graph, drive and seed as the GPU's mid line
    -- over a 100 ms prefix after the onset: the full-size CPU comparison
    for that workload (the 20 M-neuron network does not fit the oracle's
    host memory budget)."""
    import oracle
    import synth
    R, S = WORKLOAD_DIMS["mid"]
    seed = rank_seed(0, False)
    t0 = time.perf_counter()
    g = synth.make_graph([S] * R, args.k_in, seed, k_within=int(round(0.8 * args.k_in)),
                         d_within=(1, 50), d_cross=(50, 200))
    t_gen = time.perf_counter() - t0
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    s = oracle.Sim(g, params_for(args.rate, args.k_in), seed=seed + 1, precision=32, threads=threads)
    s.step(onset_steps)
    i0 = s.info()
    t0 = time.perf_counter()
    s.step(timed_steps)
    wall = time.perf_counter() - t0
    ev = s.info()["events"] - i0["events"]
    n = g.n_neurons
    del s, g
    return {"value": ev / wall, "unit": UNIT, "cores": threads, "kind": "oracle",
            "neuron_updates_per_s": n * timed_steps / wall,
            "rtf_of_sample": wall / (timed_steps * 1e-4), "cpu": cpu_model(), "generate_s": t_gen,
            "sample": "%d Euler steps (%.0f ms biological) of the full mid-size network (%s "
                      "neurons) after %d untimed steps; the matched-FP32 oracle's all-core timing "
                      "variant on %d threads" % (timed_steps, timed_steps * 0.1, f"{n:,}",
                                                 onset_steps, threads)}


# Arm "CPU part" numbers of /proc/cpuinfo (Arm's published MIDR part ids)
ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2"}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
            if line.lower().startswith("cpu part"):
                part = line.split(":", 1)[1].strip()
                return "%s (CPU part %s)" % (ARM_PARTS[part], part) if part in ARM_PARTS else part
    except OSError:
        pass
    import platform
    return platform.machine()


def run_network(args, dims, stream, dev, world, rank, seed, timed_steps, warmup, e2e_steps,
                profile_steps, pageable, clocked=True, extra_rates=()):
    """One network workload: generate, create, warm up, time `timed_steps`
    biological seconds (L2 flushed between them), time each kernel, and
    optionally the end-to-end path through the C ABI from host buffers.
    Returns the fields of a bench line."""
    import torch
    import torch.distributed as dist
    import synth
    from paper_2211_15963_gb300 import dbnet

    R, S = dims
    n_step = int(round(getattr(args, "step_ms", 1000.0) / 0.1))  # Euler steps per benchmark step
    alloc, keep = (None, None) if pageable else pinned_alloc(torch)
    t_gen = time.perf_counter()
    g = synth.make_graph([S] * R, args.k_in, seed, k_within=int(round(0.8 * args.k_in)),
                         d_within=(1, 50), d_cross=(50, 200), alloc=alloc)
    if args.two_weights:
        g = synth.with_second_weight(g, seed + 5, alloc=alloc)
    t_gen = time.perf_counter() - t_gen
    params = params_for(args.rate, args.k_in)
    opts = dict(seed=seed + 1, net_id=rank, bin_spikes=1 if args.bin_spikes else 0,
                deliver_blocks=getattr(args, "deliver_blocks", 0),
                autotune_at=getattr(args, "tune_at", 2000))

    t_create = time.perf_counter()
    net = dbnet.Network(g, params, opts, stream)
    net.sync()
    t_create = time.perf_counter() - t_create
    for _ in range(warmup):
        net.step(n_step)
    net.sync()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(timed_steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(timed_steps)]
    s0 = net.stats()
    clocks = ClockSampler(dev.index or 0) if clocked else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    wall0 = time.perf_counter()
    for k in range(timed_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        starts[k].record(stream)
        net.step(n_step)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if clocks else None
    s1 = net.stats()
    dev_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    events = s1["events"] - s0["events"]
    spikes = s1["spikes"] - s0["spikes"]
    events_all, spikes_all, neurons_all, ms_all = combine_ranks(
        events, spikes, g.n_neurons, dev_ms, world, dev)
    ms_per_step = ms_all / timed_steps

    # per-kernel device time (each kernel between CUDA events on the stream)
    p0 = net.stats()
    t_del, t_upd = net.step_timed(profile_steps)
    p1 = net.stats()
    ev_per_launch = (p1["events"] - p0["events"]) / profile_steps
    hbm, peak_kind = peaks()
    two = args.two_weights
    upd_bytes = g.n_neurons * (UPDATE_BYTES_PER_NEURON_FOUR if two else UPDATE_BYTES_PER_NEURON)
    del_bytes = ev_per_launch * (DELIVER_BYTES_PER_EVENT_TWO if two else DELIVER_BYTES_PER_EVENT)
    # a traffic summary exists only for the two standard networks
    sizes = {tuple(WORKLOAD_DIMS["large"]): "large_network", tuple(WORKLOAD_DIMS["mid"]): "mid_network"}
    name = sizes.get((g.n_regions, g.n_neurons // max(g.n_regions, 1)), "other_network")
    tag = "%s_%dhz%s" % (name, args.rate, "_two_weights" if two else "")
    kern = {
        "k_update": {"avg_us": 1e3 * t_upd / profile_steps, "algorithmic_bytes": upd_bytes,
                     "achieved_gbs": upd_bytes / (t_upd / profile_steps * 1e-3) / 1e9,
                     "traffic": measured_traffic("k_update", "traffic_%s.md" % tag)},
        "k_deliver": {"avg_us": 1e3 * t_del / profile_steps, "algorithmic_bytes": del_bytes,
                      "events_per_launch": ev_per_launch,
                      "achieved_gbs": del_bytes / (t_del / profile_steps * 1e-3) / 1e9,
                      "traffic": measured_traffic("k_deliver", "traffic_%s.md" % tag)},
    }
    for k in kern.values():
        k["frac"] = k["achieved_gbs"] / hbm
    dom = "k_update" if t_upd >= t_del else "k_deliver"
    step_bytes = upd_bytes + del_bytes
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_gbs"], "peak": hbm,
            "unit": "GB/s", "frac": kern[dom]["frac"], "traffic": kern[dom]["traffic"],
            "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "kernels": kern,
            "kernel_timing": "CUDA events around every launch on the library's stream over %d "
                             "direct (not graph-replayed) steps" % profile_steps,
            "path": {"what": "update + delivery algorithmic bytes per Euler step / the timed "
                             "graph-replayed step time (%d + %d B per neuron and event)"
                             % (UPDATE_BYTES_PER_NEURON_FOUR if two else UPDATE_BYTES_PER_NEURON,
                                DELIVER_BYTES_PER_EVENT_TWO if two else DELIVER_BYTES_PER_EVENT),
                     "achieved": step_bytes / (ms_per_step / n_step * 1e-3) / 1e9,
                     "frac": step_bytes / (ms_per_step / n_step * 1e-3) / 1e9 / hbm},
            "ncu_shape": profiled_shape()}
    stats = net.stats()
    net.close()
    del flush

    # end to end through the C ABI from host buffers: create from the host
    # graph, one biological second, stats and BOLD read, destroy
    e2e = None
    if e2e_steps > 0:
        h2d = (g.row_ptr.nbytes + 4 * g.n_edges + (4 if two else 2) * g.n_edges + g.n_edges +
               g.region_offsets.nbytes + g.n_exc.nbytes + 200 * g.n_regions)
        d2h = 8 * g.n_regions + 96
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ev_e2e = 0
        for _ in range(e2e_steps):
            h = dbnet.dbnet_create(g, params, opts, stream)
            dbnet.dbnet_step(h, STEPS_PER_BIO_S)
            st = dbnet.dbnet_stats(h)
            y = dbnet.dbnet_read_bold(h, g.n_regions, 4)
            ev_e2e += st["events"]
            dbnet.dbnet_destroy(h)
        torch.cuda.synchronize()
        t_e2e = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        ev_t = torch.tensor([float(ev_e2e)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
            dist.all_reduce(ev_t, op=dist.ReduceOp.SUM)
        e2e = {"value": float(ev_t.item()) / float(t_e2e.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "what": "dbnet_create from " + ("pageable" if pageable else "pinned") +
                       " host graph + 1 biological second + stats and "
                       "BOLD read + destroy, per step (includes the onset transient)",
               "steps": e2e_steps, "bold_samples": int(len(y))}
    out = {
        "value": events_all / (ms_all * 1e-3), "ms_per_step": ms_per_step,
        "rtf": ms_per_step / (n_step * 0.1),
        "neuron_updates_per_s": neurons_all * n_step * timed_steps / (ms_all * 1e-3),
        "mean_rate_hz": spikes_all / neurons_all / timed_steps / (n_step * 1e-4),
        "wall_s_timed": wall, "generate_s": t_gen, "create_s": t_create,
        "deliver_blocks": stats["deliver_blocks"], "segment_ring_spikes": stats["seg_ring"],
        "clocks": clk, "e2e": e2e,
        "gpu_launches": launches_per_call(n_step, SCHEDULES[stats["schedule"]]) * timed_steps,
        "schedule": SCHEDULES[stats["schedule"]],
        "roofline": roof,
    }
    # the same graph at the other mean rates: a fresh network each, one
    # biological second of warm-up (with the tuner), two timed
    if extra_rates:
        out["rates"] = {}
        r_flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for rate in extra_rates:
            r_net = None
            try:
                r_net = dbnet.Network(g, params_for(rate, args.k_in), opts, stream)
                r_net.step(n_step)
                r_net.sync()
                q0 = r_net.stats()
                r_ms = 0.0
                for _ in range(2):
                    with torch.cuda.stream(stream):
                        r_flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    r_net.step(n_step)
                    b.record(stream)
                    torch.cuda.synchronize()
                    r_ms += a.elapsed_time(b)
                q1 = r_net.stats()
                r_ev = q1["events"] - q0["events"]
                r_step = r_ms / 2
                out["rates"]["%d_hz" % rate] = {
                    "value": r_ev / (r_ms * 1e-3), "unit": UNIT, "rtf": r_step / (n_step * 0.1),
                    "mean_rate_hz": (q1["spikes"] - q0["spikes"]) / g.n_neurons / 2 / (n_step * 1e-4),
                    "steps": 2, "warmup": 1, "deliver_blocks": q1["deliver_blocks"],
                    "schedule": SCHEDULES[q1["schedule"]],
                    "path_frac": (upd_bytes + r_ev / 2 / n_step * (DELIVER_BYTES_PER_EVENT_TWO if two
                                  else DELIVER_BYTES_PER_EVENT)) / (r_step / n_step * 1e-3) / 1e9 / hbm}
            except Exception as exc:  # noqa: BLE001 -- reported in the line, the headline stands
                out["rates"]["%d_hz" % rate] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            finally:
                if r_net is not None:
                    r_net.close()
        del r_flush
    del g, keep
    return out


# -------------------------------------------------------------- our arm ----
def run_ours(args):
    import torch
    import torch.distributed as dist
    import __graft_entry__

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if local == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)  # the library and every event use this stream
    dims = workload_dims(args)
    large = dims[0] * dims[1] >= 20_000_000

    # the compact lines and the CPU sample come first: the large graph takes
    # most of the host memory once it is generated
    extras = {}
    if args.workload == "large" and not args.no_extras and world == 1:
        extras = run_extras(args, stream, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args, dims)

    # host graphs beyond 32 GB stay in pageable memory (pinning most of the
    # host's memory is not attempted)
    big_host = dims[0] * dims[1] * args.k_in * (9 if args.two_weights else 7) > 32e9
    res = run_network(args, dims, stream, dev, world, rank, rank_seed(rank, large), args.steps,
                      args.warmup, args.e2e_steps, args.profile_steps,
                      pageable=args.pageable or big_host,
                      extra_rates=tuple(r for r in (7, 30) if r != args.rate)
                      if args.workload == "large" and not args.no_extras and world == 1 else ())
    if rank == 0:
        line = {
            "metric": METRIC, "value": res.pop("value"), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators, f64 BOLD",
            "data": "synthetic (seeded generator)", "config": workload_config(args, world, dims),
        }
        line.update(res)
        line["cpu_baseline"] = cpu
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_extras(args, stream, dev):
    """Compact lines of the other workloads, measured in the same run: the
    mid-size network, the 10,000-neuron network, the batched HMDA ensemble
    and the request server, each against its own comparison."""
    out = {}
    mid_args = argparse.Namespace(**dict(vars(args), workload="mid", regions=None,
                                         region_size=None))
    m = run_network(mid_args, WORKLOAD_DIMS["mid"], stream, dev, 1, 0, rank_seed(0, False), 3, 1,
                    0, 1000, pageable=False)
    kern = m["roofline"]["kernels"]
    out["mid"] = {"config": workload_config(mid_args, 1, WORKLOAD_DIMS["mid"])["workload"],
                  "value": m["value"], "unit": UNIT, "rtf": m["rtf"], "steps": 3, "warmup": 1,
                  "mean_rate_hz": m["mean_rate_hz"], "deliver_blocks": m["deliver_blocks"],
                  "schedule": m["schedule"],
                  "k_update_us": kern["k_update"]["avg_us"], "k_update_frac": kern["k_update"]["frac"],
                  "k_deliver_us": kern["k_deliver"]["avg_us"],
                  "k_deliver_frac": kern["k_deliver"]["frac"],
                  "path_frac": m["roofline"]["path"]["frac"], "clocks": m["clocks"]}
    if not args.no_cpu_baseline:  # the oracle at full size on the host cores
        out["mid"]["cpu_baseline"] = oracle_full_mid(args)
    # the mid-size network at the paper's other two mean rates
    out["mid_rates"] = {}
    for rate in (7, 30):
        r_args = argparse.Namespace(**dict(vars(mid_args), rate=rate))
        r = run_network(r_args, WORKLOAD_DIMS["mid"], stream, dev, 1, 0, rank_seed(0, False), 2, 1,
                        0, 200, pageable=False)
        out["mid_rates"]["%d_hz" % rate] = {
            "value": r["value"], "unit": UNIT, "rtf": r["rtf"], "steps": 2, "warmup": 1,
            "mean_rate_hz": r["mean_rate_hz"], "deliver_blocks": r["deliver_blocks"],
            "schedule": r["schedule"], "path_frac": r["roofline"]["path"]["frac"],
            "clocks": r["clocks"]}
    small_args = argparse.Namespace(**dict(vars(args), steps=3, warmup=2, profile_steps=2000))
    s = run_small(small_args, stream)
    out["small"] = {k: s[k] for k in ("config", "value", "unit", "rtf", "events_per_s",
                                      "mean_rate_hz", "kernels_us", "clocks")}
    out["small"]["config"] = s["config"]["workload"]
    ens_args = argparse.Namespace(**dict(vars(args), steps=3, warmup=1, members=64, separate_trs=1))
    e = run_ensemble(ens_args, stream)
    out["batched"] = {"config": e["config"]["workload"], "value": e["value"], "unit": UNIT,
                      "trs": 3, "rtf_ensemble": e["rtf_ensemble"],
                      "analysis_ms_per_tr": e["analysis_ms_per_tr"],
                      "separate_value": e["separate"]["value"],
                      "batched_over_separate": e["batched_over_separate"],
                      "bold_fit": e["bold_fit"], "clocks": e["clocks"]}
    srv_args = argparse.Namespace(**dict(vars(args), requests=50, separate_requests=20))
    v = run_serving(srv_args, stream)
    out["served"] = {"config": v["config"]["workload"], "value": v["value"], "unit": UNIT,
                     "latency_per_bio_s": v["latency_per_bio_s"], "failed": v["failed"],
                     "saturated_value": v["saturated"]["value"],
                     "separate_value": v["separate"]["value"],
                     "separate_latency_per_bio_s": v["separate"]["latency_per_bio_s"],
                     "served_over_separate": v["served_over_separate"], "clocks": v["clocks"]}
    torch_empty_cache()
    return out


def torch_empty_cache():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# ------------------------------------------------------ ensemble workload ----
ENS_DRIVE = 3.4007   # I_ext for ~10 Hz in the 100,000-neuron, in-degree-500 network (tune_drive)
TR_MS = 800.0
TR_STEPS = 8000
LOG_LO, LOG_HI = -0.6931471805599453, 0.6931471805599453   # log 0.5, log 2


def ensemble_setup(members):
    """The batched HMDA workload: one shared 100,000-neuron graph (20 regions
    of 5,000, in-degree 500), per-member per-region AMPA and GABA_A scales
    drawn log-uniform on [0.5, 2], and a hidden member with its own draw."""
    import numpy as np
    import synth
    g = synth.ensemble_network()
    base = synth.scale_for_degree(synth.default_region_params(I_ext=ENS_DRIVE), 500)
    R = g.n_regions
    theta = np.random.default_rng(synth.seed_for(2) + 2).uniform(LOG_LO, LOG_HI, (members, R, 2))
    hidden = np.random.default_rng(synth.seed_for(2) + 3).uniform(LOG_LO, LOG_HI, (R, 2))
    return g, [dict(base) for _ in range(R)], theta, hidden


def member_params(base, th):
    """Region parameters of one member: AMPA and GABA_A conductances scaled by
    exp(theta) (the same products the ensemble forms on the device)."""
    import math
    out = []
    for r, p in enumerate(base):
        q = dict(p)
        gu = list(q["g_u"])
        gu[0] = gu[0] * math.exp(th[r, 0])
        gu[2] = gu[2] * math.exp(th[r, 1])
        q["g_u"] = tuple(gu)
        out.append(q)
    return out


def run_ensemble(args, stream=None):
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = stream or torch.cuda.Stream(dev)
    M = args.members
    g, base, theta, hidden_th = ensemble_setup(M)
    R = g.n_regions
    seed = synth.seed_for(2) + 1
    opts = dict(seed=seed, tr_ms=TR_MS, z_scale=50.0)
    enkf = dict(obs_var=1e-9, gamma=0.7, rw_sigma=0.01, theta_lo=LOG_LO, theta_hi=LOG_HI)
    n_tr = args.warmup + args.steps

    # observations: the hidden member's BOLD at every TR (not timed)
    hidden = dbnet.Network(g, member_params(base, hidden_th), dict(opts, net_id=1 << 20), stream)
    y_obs = []
    for _ in range(n_tr):
        hidden.step(TR_STEPS)
        y_obs.append(hidden.bold()[-1].copy())
    hidden.close()

    # batched: every member in each launch, one analysis per TR
    ens = dbnet.Ensemble(g, base, M, theta, dict(opts, net_id=0), enkf, stream)
    err0 = float(np.abs(theta[:, :, 0].mean(0) - hidden_th[:, 0]).mean())
    y_pred = []  # the forecast ensemble mean of every TR, before its analysis
    for k in range(args.warmup):
        ens.step(TR_STEPS)
        y_pred.append(ens.assimilate(y_obs[k]))
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    s0 = ens.stats()
    clocks = ClockSampler(0)
    clocks.start()
    for k in range(args.steps):
        ev[k][0].record(stream)
        ens.step(TR_STEPS)
        ev[k][1].record(stream)
        y_pred.append(ens.assimilate(y_obs[args.warmup + k]))  # reads the forecast mean back
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    s1 = ens.stats()
    sim_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    an_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    tot_ms = sim_ms + an_ms
    events = s1["events"] - s0["events"]
    spikes = s1["spikes"] - s0["spikes"]
    th_now, _, _ = ens.read()
    err1 = float(np.abs(th_now[:, :, 0].mean(0) - hidden_th[:, 0]).mean())
    ens.close()
    # fit of the forecast BOLD to the hidden member's (per-region correlation
    # over the TRs, and the relative error early and late)
    yp, yo = np.array(y_pred), np.array(y_obs[:len(y_pred)])
    pcc = [float(np.corrcoef(yp[:, r], yo[:, r])[0, 1]) for r in range(R) if yo[:, r].std() > 0]
    rel = np.abs(yp - yo).mean(axis=1) / np.abs(yo).mean(axis=1)
    q = max(1, len(rel) // 4)
    bold_fit = {"pcc_mean_over_regions": float(np.mean(pcc)) if pcc else None,
                "rel_err_first_quarter": float(rel[:q].mean()),
                "rel_err_last_quarter": float(rel[-q:].mean()), "trs": int(len(rel))}

    # one network per launch: the same members as independent networks,
    # stepped one after another, each from its own captured graph
    sep = []
    for m in range(M):
        sep.append(dbnet.Network(g, member_params(base, theta[m]), dict(opts, net_id=m), stream))
    for net in sep:
        net.step(TR_STEPS)          # past the onset and the autotuner, like the batched warm-up
    torch.cuda.synchronize()
    e0 = sum(n.stats()["events"] for n in sep)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.separate_trs):
        for net in sep:
            net.step(TR_STEPS)
    b.record(stream)
    torch.cuda.synchronize()
    sep_ms = a.elapsed_time(b)
    sep_events = sum(n.stats()["events"] for n in sep) - e0
    for net in sep:
        net.close()

    value = events / (tot_ms * 1e-3)
    sep_value = sep_events / (sep_ms * 1e-3)
    bio_s = args.steps * TR_MS * 1e-3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators, f64 BOLD and EnKF",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "HMDA ensemble: %d members x 100,000 neurons (20 regions x 5,000, "
                               "in-degree 500), TR 800 ms, one FP64 diffusion-EnKF analysis per "
                               "TR against a hidden member's BOLD" % M,
                   "members": M, "neurons_per_member": g.n_neurons, "regions": R,
                   "in_degree": 500, "dt_ms": 0.1, "step": "one TR (8,000 Euler steps + analysis)",
                   "l2": "not flushed: edges (300 MB) and state (370 MB) exceed L2"},
        "rtf_ensemble": tot_ms / 1e3 / bio_s,
        "neuron_updates_per_s": M * g.n_neurons * TR_STEPS * args.steps / (tot_ms * 1e-3),
        "mean_rate_hz": spikes / (M * g.n_neurons) / bio_s,
        "analysis_ms_per_tr": an_ms / args.steps, "simulate_ms_per_tr": sim_ms / args.steps,
        "theta_ampa_mean_abs_err": {"start": err0, "end": err1, "trs": n_tr},
        "bold_fit": bold_fit,
        "separate": {"value": sep_value, "unit": UNIT, "ms_per_tr": sep_ms / args.separate_trs,
                     "what": "the same %d members as independent networks, one network's "
                             "kernels per launch, stepped one after another (simulation only, "
                             "no analysis)" % M},
        "batched_over_separate": value / sep_value,
        "clocks": clk, "gpu_launches": args.steps * (2 * TR_STEPS + 14),
    }
    return line


# ------------------------------------------------------- serving workload ----
# I_ext giving ~10 Hz at in-degree K (tune_drive on 50,000-neuron, 5-region
# networks), interpolated linearly in log K -- log I_ext
SERVE_DRIVE = [(100, 0.75084), (300, 2.36363), (1000, 4.88653)]


def serve_drive(k):
    import math
    pts = SERVE_DRIVE
    if k <= pts[0][0]:
        return pts[0][1]
    for (k0, v0), (k1, v1) in zip(pts, pts[1:]):
        if k <= k1:
            t = (math.log(k) - math.log(k0)) / (math.log(k1) - math.log(k0))
            return math.exp(math.log(v0) + t * (math.log(v1) - math.log(v0)))
    return pts[-1][1]


def serving_trace(args):
    """Poisson arrivals of requests drawn from the request distribution (size
    log-uniform in [1e4, 1e6], in-degree U[100, 1000], 1-50 regions, 0.5-5 s
    biological; the within-region share of the in-degree is capped at the
    smallest region's size - 1).  To bound host generation time the networks come from a
    catalogue of `--catalogue` draws built first; each request takes one of
    them at random, with its own seed, net_id, drive and duration, and
    uploads its own copy."""
    import numpy as np
    import synth
    rng = np.random.default_rng(synth.seed_for(3))
    cat = []
    for i in range(args.catalogue):
        d = synth.serving_request(rng)
        # 80 % of the in-degree within the region, at most the region's size - 1
        kw = min(int(round(0.8 * d["k_in"])), min(d["sizes"]) - 1)
        g = synth.make_graph(d["sizes"], d["k_in"], d["seed"], k_within=kw, d_within=(1, 50),
                             d_cross=(50, 200))
        p = synth.scale_for_degree(synth.default_region_params(I_ext=serve_drive(d["k_in"])), d["k_in"])
        cat.append((g, [dict(p) for _ in d["sizes"]], d["k_in"]))
    t = 0.0
    reqs = []
    for i in range(args.requests):
        t += float(rng.exponential(1.0 / args.arrival_hz))
        c = int(rng.integers(0, len(cat)))
        bio_s = float(rng.uniform(0.5, 5.0))
        reqs.append(dict(at=t, cat=c, n_steps=int(round(bio_s * STEPS_PER_BIO_S)), bio_s=bio_s,
                         seed=int(rng.integers(1, 2**31)), net_id=i))
    return cat, reqs


def run_serving(args, stream=None):
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = stream or torch.cuda.Stream(torch.device("cuda", 0))
    t_gen = time.perf_counter()
    cat, reqs = serving_trace(args)
    t_gen = time.perf_counter() - t_gen
    srv = dbnet.Server(stream, max_neurons=8 << 20, max_requests=64, max_regions=4096,
                       max_delay=200, chunk_steps=256, arena_bytes=96 << 30)
    ids = [None] * len(reqs)
    st = [None] * len(reqs)
    pending = set()
    clocks = ClockSampler(0)
    clocks.start()
    ev0 = srv.stats()["events"]
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(reqs) or pending:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["at"] <= now:
            r = reqs[nxt]
            g, p, _ = cat[r["cat"]]
            ids[nxt] = srv.submit(g, p, r["n_steps"], seed=r["seed"], net_id=r["net_id"])
            pending.add(nxt)
            nxt += 1
        if not pending:
            time.sleep(max(0.0, min(0.002, reqs[nxt]["at"] - now)))
            continue
        stats = srv.pump()
        for i in list(pending):
            s = srv.poll(ids[i])
            if s["state"] in (dbnet.DBSRV_DONE, dbnet.DBSRV_FAILED):
                st[i] = s
                pending.discard(i)
                srv.release(ids[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    s_end = srv.stats()
    events = s_end["events"] - ev0
    launches = 2 * s_end["iterations"]

    # capacity: the first --separate-requests requests submitted at once
    n_sep = min(args.separate_requests, len(reqs))
    e1 = srv.stats()["events"]
    t1 = time.perf_counter()
    sat = []
    for r in reqs[:n_sep]:
        g, p, _ = cat[r["cat"]]
        sat.append(srv.submit(g, p, r["n_steps"], seed=r["seed"], net_id=r["net_id"]))
    srv.drain()
    torch.cuda.synchronize()
    sat_wall = time.perf_counter() - t1
    sat_events = srv.stats()["events"] - e1
    srv.close()
    failed = sum(1 for s in st if s["state"] != dbnet.DBSRV_DONE)
    lat = np.array([s["latency_s"] / r["bio_s"] for s, r in zip(st, reqs)])
    q = np.array([s["queued_s"] for s in st])
    value = events / wall

    # one network per launch: the same first requests, each created,
    # stepped and read alone; their service times then replayed through a
    # FIFO queue with the same arrival times
    service = []
    sep_events = 0
    for r in reqs[:n_sep]:
        g, p, _ = cat[r["cat"]]
        torch.cuda.synchronize()
        a = time.perf_counter()
        net = dbnet.Network(g, p, dict(seed=r["seed"], net_id=r["net_id"]), stream)
        net.step(r["n_steps"])
        sep_events += net.stats()["events"]
        net.bold()
        net.close()
        service.append(time.perf_counter() - a)
    end = 0.0
    sep_lat = []
    for r, sv in zip(reqs[:n_sep], service):
        end = max(end, r["at"]) + sv
        sep_lat.append((end - r["at"]) / r["bio_s"])
    sep_lat = np.array(sep_lat)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(reqs),
        "warmup": 0, "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators, f64 BOLD",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "serving: %d requests, Poisson arrivals at %.1f/s, networks of "
                               "1e4-1e6 neurons (log-uniform), in-degree 100-1000, 1-50 regions, "
                               "0.5-5 s biological, ~10 Hz; %d catalogue networks, each request "
                               "uploads its own copy" % (len(reqs), args.arrival_hz, args.catalogue),
                   "step": "one request", "l2": "not flushed: resident edges exceed L2"},
        "latency_per_bio_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "mean": float(lat.mean())},
        "queue_s": {"p50": float(np.percentile(q, 50)), "p99": float(np.percentile(q, 99))},
        "failed": failed, "wall_s": wall, "generate_s": t_gen,
        "separate": {"value": sep_events / sum(service), "unit": UNIT, "requests": n_sep,
                     "latency_per_bio_s": {"p50": float(np.percentile(sep_lat, 50)),
                                           "p99": float(np.percentile(sep_lat, 99))},
                     "what": "the first %d requests, each as its own network (create, step, read, "
                             "destroy) one after another; latency from their measured service "
                             "times in a FIFO queue with the same arrivals" % n_sep},
        "saturated": {"value": sat_events / sat_wall, "unit": UNIT, "requests": n_sep,
                      "what": "the same first %d requests submitted at once and drained "
                              "(capacity of the served form)" % n_sep},
        "served_over_separate": (sat_events / sat_wall) / (sep_events / sum(service)),
        "clocks": clk, "gpu_launches": launches,
    }
    return line


# ----------------------------------------------- NEST-comparison workload ----
# Supplementary Section 5 / Table 4: networks of 2-10 M neurons, in-degree
# ~100, Euler step 1 ms, mean rates ~4.1 and ~12.1 Hz, 3 s simulated and the
# last second timed.  The paper's model has no synaptic delay beyond Eq. 3's
# one step, so every edge here has delay 1.  With dt = 1 ms the conductances
# tuned for 0.1 ms make the explicit step stiff, so they are scaled by 0.2 and
# the drive set for the two rates (a sweep on a 200,000-neuron network:
# 4.13 and 12.08 Hz).
NEST_SIZES_M = (2, 3, 4, 5, 10)
NEST_G_SCALE = 0.2
NEST_DRIVE = {4.1: 0.55, 12.1: 0.9}
# Supplementary Table 4, one GPU, single precision: RTF at 2/3/4/5/10 M
NEST_PAPER_RTF = {4.1: (4.49, 6.02, 7.49, 9.18, 17.79), 12.1: (7.99, 6.28, 7.82, 17.05, 24.32)}


def run_nest(args, stream=None):
    import torch
    import synth
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = stream or torch.cuda.Stream(torch.device("cuda", 0))
    table = []
    clocks = ClockSampler(0)
    clocks.start()
    for i, n_m in enumerate(NEST_SIZES_M):
        g = synth.make_graph([20000] * (50 * n_m), 100, synth.seed_for(5) + i, d_within=(1, 1),
                             d_cross=(1, 1))
        for rate, drive in NEST_DRIVE.items():
            p = synth.default_region_params(I_ext=drive)
            p["g_u"] = tuple(x * NEST_G_SCALE for x in p["g_u"])
            net = dbnet.Network(g, p, dict(dt_ms=1.0, bin_ms=1.0, seed=synth.seed_for(5) + 100 + i),
                                stream)
            net.step(2000)
            net.sync()
            s0 = net.stats()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.step(1000)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            s1 = net.stats()
            net.close()
            table.append({"neurons": g.n_neurons, "target_hz": rate,
                          "rate_hz": (s1["spikes"] - s0["spikes"]) / g.n_neurons,
                          "rtf": ms / 1e3,
                          "events_per_s": (s1["events"] - s0["events"]) / (ms * 1e-3),
                          "paper_rtf_one_gpu": NEST_PAPER_RTF[rate][i]})
        del g
    clk = clocks.stop()
    big = [t for t in table if t["neurons"] == 10_000_000 and t["target_hz"] == 12.1][0]
    line = {
        "metric": "real-time factor", "value": big["rtf"], "unit": "s per biological s",
        "n_gpus": 1, "steps": 1, "warmup": 2, "ms_per_step": big["rtf"] * 1e3,
        "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "NEST-comparison networks: 2/3/4/5/10 M neurons, regions of "
                               "20,000, in-degree 100, delay 1 step, dt 1 ms, ~4.1 and ~12.1 Hz; "
                               "3 s simulated, the last second timed; value = 10 M at 12.1 Hz",
                   "step": "the timed biological second"},
        "table": table, "clocks": clk, "gpu_launches": 2 * 1000 * len(table),
        "paper_context": "Supplementary Table 4: one GPU with 16 GB HBM2 (10.8 TFLOPS), "
                         "their own connectome-derived networks",
    }
    return line


# ------------------------------------------------------ small network ----
def run_small(args, stream=None):
    """The 10,000-neuron network (one region, in-degree 100, delays 1-20
    steps, 10 Hz Poisson drive per neuron).  Its working set (~2 MB of state,
    6 MB of edges) stays in the L2, so the step is bound by launch and
    kernel latency, and the figures are microseconds per step and the
    real-time factor rather than a fraction of HBM bandwidth."""
    import torch
    import synth
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = stream or torch.cuda.Stream(torch.device("cuda", 0))
    g = synth.small_network()
    p = synth.default_region_params()
    net = dbnet.Network(g, p, dict(seed=synth.seed_for(0) + 1), stream)
    for _ in range(args.warmup):
        net.step(STEPS_PER_BIO_S)
    net.sync()
    s0 = net.stats()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        net.step(STEPS_PER_BIO_S)
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    s1 = net.stats()
    t_del, t_upd = net.step_timed(args.profile_steps)
    net.close()
    n_steps = STEPS_PER_BIO_S * args.steps
    line = {
        "metric": "microseconds per Euler step", "value": 1e3 * ms / n_steps, "unit": "us/step",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators, f64 BOLD",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "small network: 10,000 neurons (8,000 E / 2,000 I), one region, "
                               "in-degree 100, delays 1-20 steps, dt 0.1 ms, 10 Hz drive",
                   "step": "1 biological second (10,000 Euler steps)",
                   "l2": "resident (the whole working set fits in the L2)"},
        "rtf": ms / args.steps / 1e3,
        "events_per_s": (s1["events"] - s0["events"]) / (ms * 1e-3),
        "mean_rate_hz": (s1["spikes"] - s0["spikes"]) / g.n_neurons / args.steps,
        "kernels_us": {"k_deliver": 1e3 * t_del / args.profile_steps,
                       "k_update": 1e3 * t_upd / args.profile_steps},
        "clocks": clk, "gpu_launches": 2 * n_steps,
    }
    return line


# ------------------------------------------- step-size accuracy study ----
DT_STUDY_MS = (1.0, 0.5, 0.2, 0.1, 0.05, 0.02, 0.01, 0.008)   # the last is the reference
DT_STUDY_STEPS = 1000   # 1 ms samples of V: one biological second


def dt_study_network(dt_ms, seed):
    """The 1,000-neuron network of the step-size study: one region, in-degree
    100, every delay 1 ms (1/dt steps), the 1 ms-step conductances of the
    NEST-comparison workload and a constant injected current with no random
    drive, so that runs at different steps differ only by the Euler step."""
    import dataclasses
    import numpy as np
    import synth
    g = synth.make_graph([1000], 100, seed, d_within=(1, 1))
    d = int(round(1.0 / dt_ms))
    g = dataclasses.replace(g, delay=(np.asarray(g.delay, dtype=np.int64) * d).astype(np.uint8),
                            max_delay=d)
    p = synth.default_region_params(I_ext=NEST_DRIVE[12.1], drive_rate_hz=0.0)
    p["g_u"] = tuple(x * NEST_G_SCALE for x in p["g_u"])
    return g, p, d


def matched_spikes(ref_t, ref_i, t, i, tol):
    """Reference spikes (times ref_t of neurons ref_i) that have a spike of the
    same neuron in (t, i) within tol."""
    import numpy as np
    hit = 0
    for n in np.unique(ref_i):
        a = ref_t[ref_i == n]
        b = np.sort(t[i == n])
        if len(b) == 0:
            continue
        k = np.searchsorted(b, a)
        lo = b[np.clip(k - 1, 0, len(b) - 1)]
        hi = b[np.clip(k, 0, len(b) - 1)]
        hit += int((np.minimum(np.abs(a - lo), np.abs(hi - a)) <= tol).sum())
    return hit


def dt_study_table(runs):
    """The study's comparison.  runs[dt] = (V [ms][neuron] sampled every
    millisecond, spike times in ms, spike neuron ids, wall seconds); the
    last step of DT_STUDY_MS is the reference.  Relative error = mean over
    neurons of |V_dt - V_ref| / |V_ref|, averaged over the samples of a
    window."""
    import numpy as np
    Vr, tr_, ir, _ = runs[DT_STUDY_MS[-1]]
    n_ms = Vr.shape[0]
    table = []
    for dt in DT_STUDY_MS:
        V, ts, ids, wall = runs[dt]
        per_ms = (np.abs(V - Vr) / np.abs(Vr)).mean(axis=1)
        hit = matched_spikes(tr_, ir, ts, ids, 1.0)
        table.append({"dt_ms": dt, "rel_err_mean_1s": float(per_ms.mean()),
                      "rel_err_at_1ms": float(per_ms[0]),
                      "rel_err_mean_first_10ms": float(per_ms[:10].mean()),
                      "rel_err_mean_first_100ms": float(per_ms[:100].mean()),
                      "rel_err_mean_first_800ms": float(per_ms[:800].mean()),
                      "rel_err_at_1s": float(per_ms[-1]),
                      "rate_hz": len(ids) / Vr.shape[1] / (n_ms / 1000.0),
                      "reference_spikes_matched_within_1ms": hit / max(len(ir), 1),
                      "wall_s": wall})
    return table


def run_dt_study(args, stream=None):
    """Extended Data Fig. 1: membrane potentials of a 1,000-neuron LIF network
    integrated by forward Euler at several steps, against the finest step
    the device's 8-bit refractory counters allow (Tref = 2 ms in 250 steps).
    V of every neuron is sampled every millisecond for one second; the
    initial V (Philox counter of step 0) is the same at every step."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = stream or torch.cuda.Stream(torch.device("cuda", 0))
    seed = synth.seed_for(7)
    runs = {}
    for dt in DT_STUDY_MS:
        g, p, d = dt_study_network(dt, seed)
        net = dbnet.Network(g, p, dict(dt_ms=dt, bin_ms=1.0, seed=seed + 1,
                                       raster_capacity=1 << 22), stream)
        V = np.empty((DT_STUDY_STEPS, g.n_neurons), dtype=np.float64)
        t0 = time.perf_counter()
        for ms in range(DT_STUDY_STEPS):
            net.step(d)
            V[ms] = net.state()[0]
        wall = time.perf_counter() - t0
        st, ids = net.spikes()
        net.close()
        runs[dt] = (V, (st.astype(np.int64) + 1) * dt, ids, wall)   # spike times in ms
    table = dt_study_table(runs)
    coarse = table[0]
    line = {
        "metric": "relative membrane-potential error, dt 1 ms vs %g ms" % DT_STUDY_MS[-1],
        "value": coarse["rel_err_mean_1s"], "unit": "mean |dV| / |V| over neurons and 1 ms "
                                                     "samples of one second",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "step-size study (Extended Data Fig. 1): 1,000 neurons, in-degree "
                               "100, delays 1 ms, constant injected current, no random drive; "
                               "dt %s ms" % ", ".join("%g" % x for x in DT_STUDY_MS),
                   "reference_dt_ms": DT_STUDY_MS[-1]},
        "table": table,
        "paper_context": "Extended Data Fig. 1 / Results: about 5 % relative membrane-potential "
                         "error at dt 1 ms against 0.001 ms over one second",
        "gpu_launches": int(sum(2 * DT_STUDY_STEPS * round(1.0 / x) for x in DT_STUDY_MS)),
    }
    return line


# ------------------------------------------------- micro-column workload ----
def run_columns(args, stream=None):
    """Cortical micro-column network (Extended Data Table 3): 100 voxels of
    20,000 neurons in ten layer populations, mean in-degree 1,000 with a
    heavy-tailed out-degree; the drive is bisected for ~15 Hz on a 5-voxel
    sub-network first.  One step = one biological second, as the default
    workload, for comparison with its uniform-degree network."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet, tune

    __graft_entry__.build()
    torch.cuda.set_device(0)
    stream = stream or torch.cuda.Stream(torch.device("cuda", 0))
    base = synth.scale_for_degree(synth.default_region_params(), 1000)
    sub = synth.cortical_columns(5, 20000, 1000, seed=synth.seed_for(6) + 1)
    drive, rate_sub, _ = tune.tune_drive(sub, base, float(args.rate), knob="I_ext", lo=0.5,
                                         hi=40.0, sim_ms=300, measure_ms=200, stream=stream)
    del sub
    t_gen = time.perf_counter()
    g = synth.cortical_columns(args.regions, 20000, 1000, seed=synth.seed_for(6))
    t_gen = time.perf_counter() - t_gen
    deg = np.diff(g.row_ptr)
    p = dict(base, I_ext=drive)
    net = dbnet.Network(g, p, dict(seed=synth.seed_for(6) + 2), stream)
    for _ in range(args.warmup):
        net.step(STEPS_PER_BIO_S)
    net.sync()
    s0 = net.stats()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        net.step(STEPS_PER_BIO_S)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    s1 = net.stats()
    t_del, t_upd = net.step_timed(args.profile_steps)
    net.close()
    events = s1["events"] - s0["events"]
    line = {
        "metric": METRIC, "value": events / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 state, bf16 weights, int32 fixed-point accumulators, f64 BOLD",
        "data": "synthetic (seeded generator)",
        "config": {"workload": "cortical micro-columns: %d voxels x 20,000 neurons in ten layer "
                               "populations (Extended Data Table 3), mean in-degree 1,000, "
                               "heavy-tailed out-degree, dt 0.1 ms, ~%d Hz" % (args.regions, args.rate),
                   "step": "1 biological second"},
        "rtf": ms / args.steps / 1e3,
        "mean_rate_hz": (s1["spikes"] - s0["spikes"]) / g.n_neurons / args.steps,
        "drive_I_ext": drive, "sub_network_rate_hz": rate_sub,
        "out_degree": {"max": int(deg.max()), "p99": float(np.percentile(deg, 99)),
                       "median": float(np.median(deg))},
        "kernels_us": {"k_deliver": 1e3 * t_del / args.profile_steps,
                       "k_update": 1e3 * t_upd / args.profile_steps},
        "generate_s": t_gen, "gpu_launches": 2 * STEPS_PER_BIO_S * args.steps,
    }
    return line


# -------------------------------------------------------- reference arm ----
def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (its all-core timing
    variant; results identical to the single-threaded loop): each step is a
    10 ms (100 Euler steps) sample of a 1/20-scale network of the workload
    (a twentieth of the regions, same region size, in-degree and drive)
    after 500 untimed steps.  Under torchrun only rank 0 works."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    synth.build()
    R, S = workload_dims(args)
    r_s = max(1, R // 20)
    g = synth.make_graph([S] * r_s, args.k_in, synth.seed_for(1) + 100,
                         k_within=int(round(0.8 * args.k_in)) if r_s > 1 else args.k_in,
                         d_within=(1, 50), d_cross=(50, 200))
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    s = oracle.Sim(g, params_for(args.rate, args.k_in), seed=synth.seed_for(1) + 1, precision=32,
                   threads=threads, bin_spikes=args.bin_spikes)
    s.step(500)
    for _ in range(args.warmup):
        s.step(100)
    i0 = s.info()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(100)
    wall = time.perf_counter() - t0
    i1 = s.info()
    ev = i1["events"] - i0["events"]
    value = ev / wall
    cfg = workload_config(args, world, (r_s, S))
    cfg["workload"] = ("1/20-scale CPU sample of the %s (%s neurons): %s neurons, %d regions x %s, "
                       "in-degree %s, dt 0.1 ms, ~%d Hz"
                       % (network_name(R * S), f"{R * S:,}", f"{r_s * S:,}", r_s, f"{S:,}",
                          f"{args.k_in:,}", args.rate))
    cfg["step"] = "100 Euler steps (10 ms biological)"
    sample = ("%d x 100 Euler steps (10 ms biological each) of a %s-neuron 1/20-scale network "
              "(%d regions x %s, in-degree %s) after 500 untimed steps; the matched-FP32 oracle's "
              "all-core timing variant on %d threads (%s)"
              % (args.steps, f"{g.n_neurons:,}", r_s, f"{S:,}", f"{args.k_in:,}", threads,
                 cpu_model()))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (op-order-matched oracle)", "data": "synthetic (seeded generator)",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    runners = {"ensemble": run_ensemble, "serving": run_serving, "nest": run_nest,
               "columns": run_columns, "dt-study": run_dt_study, "small": run_small}
    if args.workload in runners:
        print(json.dumps(runners[args.workload](args)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

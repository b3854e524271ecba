#!/usr/bin/env python3
"""Benchmark of the plotting path on GB300: one JSON line on stdout.

Default workload: plain single plot K=31 (2^31 uint32 nonces, 32-byte key
from seed 31): keyed-BLAKE3 Table 1, two-level bucketing scatter, partition
sort, match and pair hashing into Table 2, both tables resident in HBM.  A
step is one whole plot (vx_table1 + vx_match); `value` is nonces/s over the
timed steps (max over ranks; weak scaling: every rank plots its own keys).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--K 31] [--impl ours|reference]

`--impl reference` times the CPU oracle (the test oracle, as it stands) on
the host cores on a bounded sample of the same workload (one K=22 plot per
step) and reports the same metric.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Blake3 nonces/s and K=31 plot seconds on 1 GB300; % INT/HBM roofline; batched vs plain"
UNIT = "nonces/s"
SMSP_PER_SM = 4
LANES = 32
# Algorithmic 32-bit integer operations of one keyed BLAKE3 compression as
# the plotter needs it: 53 message-dependent G functions x 12 ops (4 adds,
# 4 xors, 4 rotates), minus 14 ops of the last round that do not reach
# output words 0..1, plus the 2 output xors.
INT_OPS_PER_COMPRESSION = 53 * 12 - 14 + 2
KERNELS = ["key_setup", "hash_staged", "hash_direct", "scatter2", "scan_counts", "sort",
           "scan_pairs", "match", "sortmatch", "pairhash"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return {"hbm_gbs": float(m["hbm_gbs"]), "sm_max_mhz": float(m.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def device_sms(device=0) -> int:
    """Streaming multiprocessors of the CUDA device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def int_peak_ops(sm_mhz: float, sms: int) -> float:
    """Integer-issue peak: every SM sub-partition issues one 32-lane warp
    instruction per clock (SMs x 4 x 32 lanes x clock)."""
    return sms * SMSP_PER_SM * LANES * sm_mhz * 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="vx_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def free_port() -> int:
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def spawn_ranks(nproc: int, argv: list[str], env: dict | None = None) -> int:
    """Runs the python script argv[0] with arguments argv[1:] as nproc ranks
    on this node (torch.distributed.run, rendezvous on 127.0.0.1, one process
    per GPU; each reads RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from its
    environment).  Returns the launcher's exit code (non-zero if any rank
    failed)."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(nproc), "--master-addr", "127.0.0.1",
           "--master-port", str(free_port()), *argv]
    return subprocess.call(cmd, env=env)


def rank_env():
    """(world, rank, local rank) of this process, from the launcher's env."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value: float, world: int, device) -> float:
    """Max of `value` over the ranks of the default process group (the
    bench's only collective: its timing)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(nonces_per_rank: int, steps: int, ms_total_local: float, world: int, device):
    """(value in nonces/s, ms per step): every rank plots its own keys (weak
    scaling), the job's time is the slowest rank's."""
    ms_total = reduce_max(ms_total_local, world, device)
    return nonces_per_rank * steps * world / (ms_total / 1000.0), ms_total / steps


def source_digest(files) -> str:
    """Digest of the kernels' code: C/C++ comments and blank lines are dropped,
    so a comment edit does not void counters taken on the same code."""
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


_H = "paper_2606_14007_gb300/csrc/vx_internal.cuh"
KERNEL_SOURCES = {
    "hash_staged": ["paper_2606_14007_gb300/csrc/k_hash.cu", _H],
    "hash_direct": ["paper_2606_14007_gb300/csrc/k_hash.cu", _H],
    "scatter2": ["paper_2606_14007_gb300/csrc/k_sort.cu", _H],
    "sort": ["paper_2606_14007_gb300/csrc/k_sortmatch.cu", _H],
    "sortmatch": ["paper_2606_14007_gb300/csrc/k_sortmatch.cu", _H],
    "pairhash": ["paper_2606_14007_gb300/csrc/k_hash.cu", _H],
    "match": ["paper_2606_14007_gb300/csrc/k_match.cu", _H],
}


def ncu_entry(kernel: str, K: int):
    """The committed ncu figures of `kernel` at this workload, or None if absent
    or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            e = json.load(f)[kernel]
        if e.get("source_digest") != source_digest(KERNEL_SOURCES[kernel]) or int(e["K"]) != K:
            return None
        return e
    except Exception:
        return None


def ncu_traffic(kernel: str, K: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary."""
    e = ncu_entry(kernel, K)
    return float(e["bytes_per_launch"]) if e else None


def cpu_baseline(K_sample: int = 24, K_single: int = 20):
    """The CPU oracle, as it stands, on the host cores: one plot of
    2^K_sample nonces with every stage on all cores (its all-core variant:
    threaded hashing, grouped threaded sort, match over runs of whole
    buckets), and one plot of 2^K_single nonces with the plain oracle on one
    core."""
    from oracle import oracle as orc
    from paper_2606_14007_gb300.inputs import plot_key
    orc.build()
    threads = os.cpu_count() or 1
    key = plot_key(1000 + K_sample)
    t0 = time.perf_counter()
    orc.plot_allcores(K_sample, key, threads)
    dt = time.perf_counter() - t0
    key = plot_key(1000 + K_single)
    t0 = time.perf_counter()
    orc.plot(K_single, key)
    dt1 = time.perf_counter() - t0
    return {"value": (1 << K_sample) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "one K=%d plot (2^%d nonces) with every stage (hash, sort, match incl. pair "
                      "hashing) on all %d host cores; %.1f s" % (K_sample, K_sample, threads, dt),
            "single_thread": {"value": (1 << K_single) / dt1, "unit": UNIT, "cores": 1,
                              "sample": "one K=%d plot entirely on 1 thread (plain oracle); %.1f s"
                                        % (K_single, dt1)}}


def run_reference(args):
    """CPU oracle as the reference arm: one K=22 plot per step, every stage
    on all host cores (the oracle's all-core variant)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    from paper_2606_14007_gb300.inputs import plot_key
    orc.build()
    Ks = 22
    threads = os.cpu_count() or 1

    def step(i):
        orc.plot_allcores(Ks, plot_key(2000 + i), threads)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    value = (1 << Ks) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "plain plot, bounded sample: one K=22 plot per step on the CPU oracle",
                   "K": Ks, "key_seeds": "2000+i"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "one K=22 plot per step, every stage on %d host cores" % threads},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--K", type=int, default=31)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-copy-streams", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="plain",
                    choices=["plain", "batch", "large", "serve", "write", "sort2", "tiled", "plotfile",
                             "hashpeak", "sweep"],
                    help="plain: the K=31 headline; batch: 64 mixed-K plots batched vs plain; "
                         "large: 4 x K=29 + 8 x K=27 batched vs plain; serve: Poisson requests "
                         "through the continuous-batching server vs one at a time; write: plots "
                         "written to flat Table-2 files, serial vs overlapped with the next plot; "
                         "sort2: Table 2 of a K plot sorted by hash2; tiled: a K plot built "
                         "window by window into pinned host memory vs the whole plot and its copy; "
                         "plotfile: one K plot file end to end (plot, write, fsync), whole and tiled; "
                         "hashpeak: the hash-only ceiling (no record stores); sweep: per-K plot "
                         "times and kernel split for K=22 and 27..31 beside the oracle")
    ap.add_argument("--partition-log2", type=int, default=0)
    ap.add_argument("--scatter-mode", type=int, default=0)
    ap.add_argument("--nonces-per-thread", type=int, default=0,
                    help="Table-1 hash: 0 (= 8), 4, 8 or 16 nonces per thread")
    ap.add_argument("--fuse-pair-hash", type=int, default=0)
    ap.add_argument("--pipeline-chunks", type=int, default=0)
    ap.add_argument("--t2-placement", type=int, default=0,
                    help="0 automatic, 1 look-back, 2 pair slots")
    ap.add_argument("--match-scope", type=int, default=0,
                    help="0 pairs inside a logical bucket, 1 cross-bucket")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--sweep-oracle-max-k", type=int, default=27,
                    help="sweep: largest K of the all-core oracle timed (larger K extrapolated)")
    ap.add_argument("--sweep-oracle-1t-max-k", type=int, default=23,
                    help="sweep: largest K of the single-thread oracle timed")
    ap.add_argument("--autotune", action="store_true",
                    help="batch / large: every K plotted with the autotuner's plan (cached on disk)")
    ap.add_argument("--serve-streams", type=int, default=0, help="serve: concurrent waves (0 = library default)")
    ap.add_argument("--serve-no-plain", action="store_true",
                    help="serve: skip the one-at-a-time leg (a long latency run at a rate far below capacity)")
    ap.add_argument("--serve-max-wave", type=int, default=0, help="serve: plots per wave (0 = library default)")
    ap.add_argument("--serve-max-inflight", type=int, default=0,
                    help="serve: plots on the device at once (0 = library default)")
    ap.add_argument("--write-K", type=int, default=28, help="write: K of every plot")
    ap.add_argument("--write-plots", type=int, default=6, help="write: plots per leg")
    ap.add_argument("--write-dir", default=None, help="write: directory for the plot files")
    ap.add_argument("--window-bits", type=int, default=2, help="tiled: 2^c windows")
    ap.add_argument("--tiled-no-table1", action="store_true",
                    help="tiled: copy out Table 2 only (the plot file's table)")
    ap.add_argument("--tiled-no-whole", action="store_true",
                    help="tiled: skip the whole-plot comparison leg (e.g. when it does not fit)")
    ap.add_argument("--tiled-file", default=None,
                    help="tiled: write Table 2 as a plot file in this directory (vx_plot_tiled_write) "
                         "instead of into host memory; compared with the whole plot + vx_plot_write")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    if args.mode != "plain":
        if args.gpus != 1 or "WORLD_SIZE" in os.environ:
            ap.error("--mode %s runs on one GPU (--gpus 1, no launcher)" % args.mode)
        return run_mode(args)

    import torch
    import torch.distributed as dist

    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # Started without a launcher: run the N replica ranks ourselves, one
        # GPU each, every rank plotting its own keys (no data-path collective).
        have = torch.cuda.device_count()
        if have < args.gpus:
            print("bench.py: --gpus %d but %d CUDA device(s) visible" % (args.gpus, have),
                  file=sys.stderr)
            return 2
        return spawn_ranks(args.gpus, [os.path.abspath(__file__), *sys.argv[1:]])
    world, rank, local = rank_env()
    if world != args.gpus:
        print("bench.py: --gpus %d but the launcher started %d rank(s)" % (args.gpus, world),
              file=sys.stderr)
        return 2
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    import __graft_entry__
    if local == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2606_14007_gb300 import vaultx as vx
    from paper_2606_14007_gb300.inputs import plot_key
    vx.lib()

    K = args.K
    N = 1 << K
    key = plot_key(K + 1000 * rank)
    stream = torch.cuda.current_stream()
    plot = vx.Plot(K, key, plot_opts(vx, args))

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        plot.run(stream)
    n2 = plot.sync()

    vx.vx_plot_profile(plot.handle, args.steps)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        vx.vx_plot_run(plot.handle, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1)
    n2 = plot.sync()          # raises on any device-side status error
    per_kernel, runs = vx.vx_plot_profile_read(plot.handle)
    vx.vx_plot_profile(plot.handle, 0)
    value, ms_step = aggregate(N, args.steps, ms_local, world, "cuda")

    # Per-kernel figures (CUDA events on the launching stream, timed region).
    pk = {}
    pk_peak = peaks()
    hbm_peak = pk_peak["hbm_gbs"]
    sms = device_sms(local)
    int_peak = int_peak_ops(pk_peak["sm_max_mhz"], sms)
    # Algorithmic work per launch: a hash kernel does one compression per
    # nonce and writes 12 B per record; the second scatter level reads and
    # writes 12 B per record; sort+match reads 12 B and writes 12 B per
    # record and writes 16 B per pair (8 B with the pair slots), and hashes
    # the pairs unless the separate pair-hash pass does (it reads 16 B, or
    # 8 B from the pair slots, and writes 16 B per pair); the pair-count
    # scan reads 8 B and writes 8 B per partition.
    mask = vx.vx_plot_kernel_mask(plot.handle)
    separate = "pairhash" in mask
    slots = "scan_pairs" in mask
    pair_out = 8 if slots else 16
    algo_bytes = {"scatter2": 24 * N, "sort": 24 * N, "match": 12 * N + 16 * n2,
                  "sortmatch": 24 * N + pair_out * n2, "hash_direct": 12 * N, "hash_staged": 12 * N,
                  "pairhash": (pair_out + 16) * n2}
    algo_ops = {"hash_staged": INT_OPS_PER_COMPRESSION * N, "hash_direct": INT_OPS_PER_COMPRESSION * N,
                "match": INT_OPS_PER_COMPRESSION * n2, "pairhash": INT_OPS_PER_COMPRESSION * n2}
    if not separate:
        algo_ops["sortmatch"] = INT_OPS_PER_COMPRESSION * n2
    launched = vx.vx_plot_kernel_mask(plot.handle)
    for k in KERNELS:
        if k not in launched:
            continue
        ms = per_kernel[k] / max(1, runs)
        e = {"ms_per_launch": ms}
        if k in algo_ops and ms > 0:
            e["int_tops"] = algo_ops[k] / (ms / 1e3) / 1e12
            e["int_frac"] = e["int_tops"] * 1e12 / int_peak
        if k in algo_bytes and ms > 0:
            e["gbs"] = algo_bytes[k] / (ms / 1e3) / 1e9
            e["hbm_frac"] = e["gbs"] / hbm_peak
        pk[k] = e
    dom = max(pk, key=lambda k: pk[k]["ms_per_launch"])
    if dom in algo_ops:
        ach = pk[dom]["int_tops"] * 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach / 1e12, "peak": int_peak / 1e12,
                "unit": "Tops/s (32-bit integer)", "frac": ach / int_peak,
                "peak_basis": "%d SMs (device) x 4 sub-partitions x 32 lanes x %.0f MHz (max SM clock, %s)"
                              % (sms, pk_peak["sm_max_mhz"], pk_peak["source"]),
                "work_per_launch": algo_ops[dom],
                "traffic": ncu_traffic(dom, K)}
        ceil = hash_ceiling(vx, stream, sms)
        roof["peak_measured"] = {
            "value": ceil["int_ops_per_s"] / 1e12, "unit": "Tops/s (32-bit integer)",
            "frac": ach / ceil["int_ops_per_s"],
            "source": "vx_hash_peak in this run: the same keyed BLAKE3 in the Table-1 kernel's shape "
                      "with no record stores, 2^31 nonces, best grid of 2..16 CTAs/SM (%d), %.2f ms"
                      % (ceil["ctas_per_sm"], ceil["ms_per_2^31"])}
        ent = ncu_entry(dom, K)
        if ent and "alu_pipe_pct" in ent:
            # the integer (ALU) pipe's own occupancy, from the committed ncu
            # capture of the same kernel code
            roof["alu_pipe_busy_ncu"] = ent["alu_pipe_pct"] / 100.0
    else:
        ach = pk[dom]["gbs"]
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "work_per_launch": algo_bytes[dom],
                "traffic": ncu_traffic(dom, K)}

    # End to end through the C ABI with host buffers: per step the key goes
    # host -> device (plot descriptor upload from pinned memory) and Table 2
    # comes back device -> host (pinned), all inside the timed region.  Two
    # Table-2 buffers let plot i+1 compute while Table 2 of plot i is copied
    # out on a copy stream (Table 1 and scratch are reused plot after plot
    # on the compute stream); vx_sync waits for one plot only.
    e2e = None
    if args.e2e_steps > 0:
        chunk = 1 << 30
        nring = max(1, args.e2e_copy_streams)
        ring = torch.empty(nring * chunk, dtype=torch.uint8).pin_memory()
        t2_bufs = [plot._t2, torch.empty_like(plot._t2)]
        t2_cap = plot._t2.numel() // 16
        copy_streams = [torch.cuda.Stream() for _ in range(nring)]
        copy_done = [torch.cuda.Event(), torch.cuda.Event()]
        opts = plot_opts(vx, args)

        def copy_out(h, slot):
            _, m, _, _ = vx.vx_table_info(h, vx.VX_TABLE2)
            off, k = 0, 0
            while off < 16 * m:
                nb = min(chunk, 16 * m - off)
                cs = copy_streams[k % nring]
                vx.vx_table_copy(h, vx.VX_TABLE2, ring.data_ptr() + (k % nring) * chunk, nb, cs,
                                 offset=off)
                off += nb
                k += 1
            for cs in copy_streams[1:]:
                copy_streams[0].wait_stream(cs)
            copy_done[slot].record(copy_streams[0])
            return m

        # the box's device-to-host rate into pinned memory, which bounds e2e:
        # Table 2 (1 GiB pieces of the plot's buffer) into the ring, untimed
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        probe = min(8 * chunk, plot._t2.numel())
        with torch.cuda.stream(copy_streams[0]):
            d0.record()
            for k, off in enumerate(range(0, probe, chunk)):
                nb = min(chunk, probe - off)
                ring[(k % nring) * chunk:(k % nring) * chunk + nb].copy_(plot._t2[off:off + nb],
                                                                       non_blocking=True)
            d1.record()
        torch.cuda.synchronize()
        d2h_gbs = probe / (d0.elapsed_time(d1) / 1e3) / 1e9
        handles, counts = [], []
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for i in range(args.e2e_steps):
            slot = i % 2
            h = vx.vx_plot_create(K, plot_key(K + 1000 * rank + 1 + i), opts)
            vx.vx_plot_bind(h, plot._t1.data_ptr(), t2_bufs[slot].data_ptr(),
                            plot._scratch.data_ptr(), t2_cap)
            if i >= 2:
                stream.wait_event(copy_done[slot])
            vx.vx_plot_run(h, stream)
            if prev is not None:
                vx.vx_sync(prev)
                counts.append(copy_out(prev, (i - 1) % 2))
            handles.append(h)
            prev = h
        vx.vx_sync(prev)
        counts.append(copy_out(prev, (args.e2e_steps - 1) % 2))
        for cs in copy_streams:
            cs.synchronize()
        dt = time.perf_counter() - t0
        barrier()
        for h in handles:
            vx.vx_plot_destroy(h)
        del t2_bufs
        desc_bytes = 512
        e2e = {"value": N * args.e2e_steps * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": desc_bytes,
               "d2h_bytes_per_step": int(16 * sum(counts) / len(counts)) + 12,
               "steps": args.e2e_steps, "d2h_gbs_measured": d2h_gbs,
               "note": "per step: vx_plot_create from a host key, vx_plot_bind, vx_plot_run, "
                       "vx_sync, Table 2 copied to pinned host memory with vx_table_copy "
                       "(1 GiB pieces on %d copy stream(s)); the copy of plot i overlaps plot "
                       "i+1 (two Table-2 buffers)" % nring}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    launches_per_step = len(launched)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "plain single plot K=%d (2^%d uint32 nonces, key from seed %d), "
                               "Table 1 + Table 2 resident in HBM" % (K, K, K),
                   "K": K, "table2_records": n2,
                   "l2": "inputs larger than L2: Table 1 %.1f GB, Table 2 %.1f GB per plot"
                         % (12 * N / 1e9, 16 * n2 / 1e9)},
        "plot_seconds": ms_step / 1000.0,
        "roofline": roof,
        "kernels": pk,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    plot.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def plot_opts(vx, args):
    return vx.make_opts(partition_log2=args.partition_log2, scatter_mode=args.scatter_mode,
                        fuse_pair_hash=args.fuse_pair_hash, pipeline_chunks=args.pipeline_chunks,
                        t2_placement=args.t2_placement, match_scope=args.match_scope,
                        nonces_per_thread=args.nonces_per_thread)


def _timed(fn, stream):
    """Milliseconds of fn() on the device (CUDA events on `stream`)."""
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def hash_ceiling(vx, stream, sms: int, K: int = 31, reps: int = 3):
    """The hash-only ceiling: vx_hash_peak over 2^K nonces (no record
    stores) at grids of 2, 3, 4, 8 and 16 CTAs per SM, best of `reps` timed
    launches each after one untimed one; returns the best rate and the
    sweep."""
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    key = plot_key(K)
    N = 1 << K
    sweep = {}
    for per_sm in (2, 3, 4, 8, 16):
        words = 256 * per_sm * sms
        fold = torch.empty(words, dtype=torch.int32, device="cuda")
        vx.vx_hash_peak(key, 0, N, fold.data_ptr(), words, stream)
        best = min(_timed(lambda: vx.vx_hash_peak(key, 0, N, fold.data_ptr(), words, stream), stream)
                   for _ in range(reps))
        sweep[str(per_sm)] = best
        del fold
    per_sm, ms = min(sweep.items(), key=lambda kv: kv[1])
    ops = INT_OPS_PER_COMPRESSION * N / (ms / 1e3)
    return {"compressions_per_s": N / (ms / 1e3), "int_ops_per_s": ops, "ms_per_2^%d" % K: ms,
            "ctas_per_sm": int(per_sm), "sweep_ms": sweep}


def run_hashpeak(vx, args):
    import torch
    stream = torch.cuda.current_stream()
    sms = device_sms(int(os.environ.get("LOCAL_RANK", "0")))
    pk = peaks()
    c = hash_ceiling(vx, stream, sms, args.K)
    nominal = int_peak_ops(pk["sm_max_mhz"], sms)
    c.update({"mode": "hashpeak", "K": args.K, "sms": sms,
              "nominal_int_ops_per_s": nominal, "frac_of_nominal": c["int_ops_per_s"] / nominal,
              "note": "keyed BLAKE3 of 2^K nonces in the Table-1 kernel's shape with no record "
                      "stores (vx_hash_peak); %d int32 ops per compression" % INT_OPS_PER_COMPRESSION})
    return c


def run_sweep(vx, args):
    """Per-K results: for K = 22 and 27 .. 31 one plain plot per step (key
    from seed K), device ms per plot (CUDA events on the launching stream,
    `steps` timed after `warmup`), nonces/s, the per-kernel split, and
    T(k+1)/T(k); beside them the oracle on the host cores: single-thread
    (plain oracle) measured at K = 20 .. --sweep-oracle-1t-max-k, all cores
    (its all-core variant) at K = 20 .. --sweep-oracle-max-k, each only
    while its tables fit the free host memory; larger K extrapolated as
    N log N from the largest measured K and labelled so."""
    import torch
    from oracle import oracle as orc
    from paper_2606_14007_gb300.inputs import plot_key
    stream = torch.cuda.current_stream()
    rows = []
    for K in (22, 27, 28, 29, 30, 31):
        plot = vx.Plot(K, plot_key(K), plot_opts(vx, args))
        for _ in range(args.warmup):
            plot.run(stream)
        plot.sync()
        vx.vx_plot_profile(plot.handle, args.steps)
        ms = _timed(lambda: [vx.vx_plot_run(plot.handle, stream) for _ in range(args.steps)], stream)
        ms /= args.steps
        n2 = plot.sync()
        per_kernel, runs = vx.vx_plot_profile_read(plot.handle)
        vx.vx_plot_profile(plot.handle, 0)
        split = {k: v / max(1, runs) for k, v in per_kernel.items() if v > 0}
        rows.append({"K": K, "plot_ms": ms, "nonces_per_s": (1 << K) / (ms / 1e3),
                     "table2_records": n2, "kernel_ms": split})
        plot.close()
        del plot
        torch.cuda.empty_cache()
    for a, b in zip(rows, rows[1:]):
        if b["K"] == a["K"] + 1:
            b["ratio_vs_prev_K"] = b["plot_ms"] / a["plot_ms"]
    orc.build()
    threads = os.cpu_count() or 1
    single, allc = {}, {}

    def fits(K):
        # Table 1 and its sort scratch, then Table 1 and Table 2: at most
        # about 30 bytes per nonce at once, with a quarter of the memory spare
        try:
            free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        except (ValueError, OSError):
            return K <= 27
        return 30 * (1 << K) <= 0.75 * free

    for K in range(20, args.sweep_oracle_1t_max_k + 1):
        if not fits(K):
            break
        t0 = time.perf_counter()
        orc.plot(K, plot_key(K))
        single[K] = time.perf_counter() - t0
    for K in range(20, args.sweep_oracle_max_k + 1):
        if not fits(K):
            break
        t0 = time.perf_counter()
        orc.plot_allcores(K, plot_key(K), threads)
        allc[K] = time.perf_counter() - t0

    def est(meas, K):
        if K in meas:
            return {"s": meas[K], "measured": True}
        k0 = max(meas)
        return {"s": meas[k0] * 2 ** (K - k0) * K / k0, "measured": False}

    for r in rows:
        r["oracle_1_thread"] = est(single, r["K"])
        r["oracle_all_cores"] = est(allc, r["K"])
        r["gpu_over_oracle_all_cores"] = r["oracle_all_cores"]["s"] / (r["plot_ms"] / 1e3)
    return {"mode": "sweep", "rows": rows, "oracle_cores": threads,
            "note": "device plot time per K (vx_plot_run, tables resident in HBM); oracle seconds "
                    "with measured=false are extrapolated as N log N from the largest measured K"}


def run_batch_compare(vx, mix, steps, warmup, name, label, tune=False):
    """The same plots plotted one vx_plot_run after the other (plain) and as
    one vx_plot_batch (grouped launches in a recorded CUDA graph); every
    plot's tables must be identical both ways.  With tune, every K gets the
    autotuner's plan (both legs use the same plans)."""
    import torch
    stream = torch.cuda.current_stream()
    tuned = {}
    if tune:
        for K in sorted({K for K, _ in mix}):
            tuned[K] = vx.autotune(K)
    plots = [vx.Plot(K, key, tuned.get(K)) for K, key in mix]
    handles = [p.handle for p in plots]
    nonces = sum(1 << K for K, _ in mix)

    def plain():
        for p in plots:
            vx.vx_plot_run(p.handle, stream)

    def batched():
        vx.vx_plot_batch(handles, stream)

    for _ in range(warmup):
        plain()
    ms_plain = _timed(lambda: [plain() for _ in range(steps)], stream) / steps
    ref = []
    for p in plots:
        p.sync()
        ref.append((p.t1.clone(), p.t2.clone()) if label == "batch" else None)
    for _ in range(warmup):
        batched()
    ms_batch = _timed(lambda: [batched() for _ in range(steps)], stream) / steps
    equal = True
    for i, p in enumerate(plots):
        p.sync()
        if ref[i] is not None:
            equal = equal and torch.equal(p.t1, ref[i][0]) and torch.equal(p.t2, ref[i][1])
    if label == "large":
        # one plot at a time alone, in a separate buffer set, against the batch's tables
        for (K, key), p in zip(mix, plots):
            q = vx.Plot(K, key)
            q.run()
            q.sync()
            equal = equal and torch.equal(q.t1, p.t1) and torch.equal(q.t2, p.t2)
            q.close()
            del q
            torch.cuda.empty_cache()
    for p in plots:
        p.close()
    return {"mode": label, "metric": name, "unit": "nonces/s", "plots": len(mix),
            "nonces_per_step": nonces,
            "plain": {"value": nonces / (ms_plain / 1e3), "ms_per_step": ms_plain,
                      "how": "one vx_plot_run after the other on one stream"},
            "batched": {"value": nonces / (ms_batch / 1e3), "ms_per_step": ms_batch,
                        "how": "vx_plot_batch: grouped launches recorded into a CUDA graph"},
            "batched_over_plain": ms_plain / ms_batch, "equal_output": bool(equal),
            "autotuned": {str(K): {"partition_log2": o.partition_log2, "scatter_mode": o.scatter_mode,
                                   "nonces_per_thread": o.nonces_per_thread}
                          for K, o in tuned.items()} or None,
            "steps": steps, "warmup": warmup, "data": "synthetic"}


def run_serve(vx, args):
    """Poisson plot requests through the continuous-batching server, and the
    same requests plotted one at a time on one preallocated buffer set."""
    import numpy as np
    import torch
    from paper_2606_14007_gb300.inputs import poisson_arrivals
    arrivals = poisson_arrivals(args.rate, args.duration, 22, 29, 7)

    def pct(xs, q):
        return float(np.percentile(np.array(xs), q)) if xs else None

    # -- server
    so = None
    if args.serve_streams or args.serve_max_wave or args.serve_max_inflight:
        so = vx.vx_serve_opts()
        so.size = ctypes.sizeof(vx.vx_serve_opts)
        so.streams = args.serve_streams
        so.max_wave = args.serve_max_wave
        so.max_inflight = args.serve_max_inflight
    srv = vx.vx_serve_create(so)
    lat, done_nonces, failed = [], 0, 0
    pending = {}
    i = 0
    t0 = time.perf_counter()
    while i < len(arrivals) or pending:
        now = time.perf_counter() - t0
        while i < len(arrivals) and arrivals[i][0] <= now:
            _, K, key = arrivals[i]
            pending[vx.vx_serve_submit(srv, K, key)] = K
            i += 1
        for t in list(pending):
            st, h = vx.vx_serve_poll(srv, t)
            if st == vx.VX_DONE:
                lat.append(vx.vx_serve_latency(srv, t))
                done_nonces += 1 << pending.pop(t)
                vx.vx_plot_destroy(h)
            elif st == vx.VX_FAILED:
                failed += 1
                pending.pop(t)
        if not pending and i < len(arrivals):
            time.sleep(max(0.0, min(0.002, arrivals[i][0] - (time.perf_counter() - t0))))
    served_s = time.perf_counter() - t0
    vx.vx_serve_destroy(srv)

    if args.serve_no_plain:
        return {"mode": "serve", "metric": "plot-request latency and aggregate nonces/s",
                "unit": "nonces/s", "rate_per_s": args.rate, "duration_s": args.duration,
                "requests": len(arrivals), "K_range": [22, 29],
                "served": {"value": done_nonces / served_s, "p50_s": pct(lat, 50), "p99_s": pct(lat, 99),
                           "completed": len(lat), "failed": failed, "wall_s": served_s,
                           "how": "vx_serve_submit/poll: admission by HBM footprint"},
                "one_at_a_time": None, "data": "synthetic"}

    # -- one at a time, first come first served, on one buffer set sized for K=29
    t1b, t2b, sb = vx.vx_plot_required_bytes(29)
    b1 = torch.empty(t1b, dtype=torch.uint8, device="cuda")
    b2 = torch.empty(t2b, dtype=torch.uint8, device="cuda")
    bs = torch.empty(sb, dtype=torch.uint8, device="cuda")
    plain_lat, plain_nonces = [], 0
    t0 = time.perf_counter()
    for (t_arr, K, key) in arrivals:
        now = time.perf_counter() - t0
        if now < t_arr:
            time.sleep(t_arr - now)
        h = vx.vx_plot_create(K, key)
        vx.vx_plot_bind(h, b1.data_ptr(), b2.data_ptr(), bs.data_ptr(), 0)
        vx.vx_plot_run(h)
        vx.vx_sync(h)
        vx.vx_plot_destroy(h)
        plain_lat.append(time.perf_counter() - t0 - t_arr)
        plain_nonces += 1 << K
    plain_s = time.perf_counter() - t0
    return {"mode": "serve", "metric": "plot-request latency and aggregate nonces/s",
            "unit": "nonces/s", "rate_per_s": args.rate, "duration_s": args.duration,
            "requests": len(arrivals), "K_range": [22, 29],
            "server_opts": {"streams": args.serve_streams or "default", "max_wave": args.serve_max_wave or "default",
                            "max_inflight": args.serve_max_inflight or "default"},
            "served": {"value": done_nonces / served_s, "p50_s": pct(lat, 50), "p99_s": pct(lat, 99),
                       "completed": len(lat), "failed": failed, "wall_s": served_s,
                       "how": "vx_serve_submit/poll: admission by HBM footprint, waves on 2 streams"},
            "one_at_a_time": {"value": plain_nonces / plain_s, "p50_s": pct(plain_lat, 50),
                              "p99_s": pct(plain_lat, 99), "completed": len(plain_lat),
                              "wall_s": plain_s,
                              "how": "arrival order, vx_plot_run + vx_sync per request"},
            "data": "synthetic"}


def run_write(vx, args):
    """NEXT-1: plots of one K written as flat Table-2 files (vx_plot_write:
    D2H through pinned staging, 4 MB sequential writes), serial against
    overlapped with the next plot's kernels (two Table-2 buffers, a writer
    thread; Table 1 and scratch shared on the compute stream)."""
    import concurrent.futures as cf
    import shutil
    import tempfile
    import numpy as np
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    K, nplots = args.write_K, args.write_plots
    stream = torch.cuda.current_stream()
    t1b, t2b, sb = vx.vx_plot_required_bytes(K)
    t1 = torch.empty(t1b, dtype=torch.uint8, device="cuda")
    sc = torch.empty(sb, dtype=torch.uint8, device="cuda")
    t2 = [torch.empty(t2b, dtype=torch.uint8, device="cuda") for _ in range(2)]
    wdir = tempfile.mkdtemp(prefix="vx_plots_", dir=args.write_dir)
    paths = [os.path.join(wdir, "plot%d.bin" % i) for i in range(2)]

    def make(i):
        h = vx.vx_plot_create(K, plot_key(5000 + i))
        vx.vx_plot_bind(h, t1.data_ptr(), t2[i % 2].data_ptr(), sc.data_ptr(), t2b // 16)
        return h

    def write(h, i):
        d2h, total = vx.vx_plot_write(h, paths[i % 2])
        c0 = time.perf_counter()
        fd = os.open(paths[i % 2], os.O_RDONLY)
        os.fsync(fd)
        os.close(fd)
        return d2h, total, time.perf_counter() - c0

    try:
        # warm-up: one plot, written and checked against Table 2 on the device
        h = make(0)
        vx.vx_plot_run(h, stream)
        write(h, 0)
        _, n2, _, _ = vx.vx_table_info(h, vx.VX_TABLE2)
        got = np.fromfile(paths[0], dtype=np.uint8)
        equal = got.size == 16 * n2 and bool(
            (torch.from_numpy(got).cuda() == t2[0][: 16 * n2]).all().item())
        vx.vx_plot_destroy(h)
        file_bytes = 16 * n2

        # serial: plot, then write, one after the other
        stats = []
        t0 = time.perf_counter()
        for i in range(nplots):
            h = make(i)
            vx.vx_plot_run(h, stream)
            stats.append(write(h, i))
            vx.vx_plot_destroy(h)
        serial_s = time.perf_counter() - t0

        # overlapped: plot i+1 computes while plot i is written
        ostats = []
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=1) as ex:
            futs = []
            for i in range(nplots):
                if i >= 2:
                    ostats.append(futs[i - 2][0].result())  # frees Table-2 buffer i % 2
                    vx.vx_plot_destroy(futs[i - 2][1])
                h = make(i)
                vx.vx_plot_run(h, stream)
                futs.append((ex.submit(write, h, i), h))
            for f, h in futs[max(0, nplots - 2):]:
                ostats.append(f.result())
                vx.vx_plot_destroy(h)
        overlap_s = time.perf_counter() - t0
    finally:
        shutil.rmtree(wdir, ignore_errors=True)

    def mean(xs, k):
        return float(np.mean([x[k] for x in xs]))

    nonces = nplots * (1 << K)
    return {"mode": "write", "metric": "plots written to flat Table-2 files, nonces/s end to end",
            "unit": "nonces/s", "K": K, "plots": nplots, "file_bytes": int(file_bytes),
            "dir_fs": wdir.rsplit("/", 1)[0],
            "serial": {"value": nonces / serial_s, "s_per_plot": serial_s / nplots,
                       "d2h_s": mean(stats, 0), "write_s": mean(stats, 1), "fsync_s": mean(stats, 2),
                       "file_GBps": file_bytes / mean(stats, 1) / 1e9,
                       "how": "vx_plot_run, vx_plot_write (+ fsync), next plot"},
            "overlapped": {"value": nonces / overlap_s, "s_per_plot": overlap_s / nplots,
                           "d2h_s": mean(ostats, 0), "write_s": mean(ostats, 1),
                           "fsync_s": mean(ostats, 2),
                           "how": "writer thread runs vx_plot_write (+ fsync) of plot i while "
                                  "plot i+1 runs; two Table-2 buffers"},
            "overlapped_over_serial": serial_s / overlap_s, "equal_output": bool(equal),
            "data": "synthetic"}


def run_sort2(vx, args):
    """NEXT-3: Table 2 of a K plot sorted by hash2 (vx_sort_table2), timed
    with CUDA events; the result is checked on the device: ascending
    (key2, a, b) and the same multiset of records (sums of the words)."""
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    K = args.K
    stream = torch.cuda.current_stream()
    p = vx.Plot(K, plot_key(K), plot_opts(vx, args))
    p.run(stream)
    n2 = p.sync()
    wb = vx.vx_sort_table2_work_bytes(p.handle)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")

    def words_sum():
        acc = torch.zeros(4, dtype=torch.int64, device="cuda")
        for s in range(0, n2, 1 << 27):
            acc += p.t2[s:min(n2, s + (1 << 27))].view(torch.int32).to(torch.int64).sum(0)
        return acc.tolist()

    before = words_sum()
    for _ in range(args.warmup):
        vx.vx_sort_table2(p.handle, work.data_ptr(), wb, stream)
    ms = _timed(lambda: [vx.vx_sort_table2(p.handle, work.data_ptr(), wb, stream)
                         for _ in range(args.steps)], stream) / args.steps
    ok = vx.vx_sync(p.handle, check=False) == vx.VX_OK and words_sum() == before
    t2 = p.t2
    step = 1 << 27
    prev = None
    for s in range(0, n2, step):
        b = t2[s:min(n2, s + step)].long()
        a_ = b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16) | (b[:, 3] << 24)
        b_ = b[:, 4] | (b[:, 5] << 8) | (b[:, 6] << 16) | (b[:, 7] << 24)
        hi = (b[:, 8] << 24) | (b[:, 9] << 16) | (b[:, 10] << 8) | b[:, 11]
        lo = (b[:, 12] << 24) | (b[:, 13] << 16) | (b[:, 14] << 8) | b[:, 15]
        if prev is not None:
            a_, b_, hi, lo = (torch.cat([x, y]) for x, y in zip(prev, (a_, b_, hi, lo)))
        inc = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (
            (lo[1:] > lo[:-1]) | ((lo[1:] == lo[:-1]) & (
                (a_[1:] > a_[:-1]) | ((a_[1:] == a_[:-1]) & (b_[1:] > b_[:-1]))))))
        ok = ok and bool(inc.all())
        prev = (a_[-1:], b_[-1:], hi[-1:], lo[-1:])
    pk = peaks()
    algo = 96 * n2  # two scatter levels and the sort, each reads and writes 16 B per record
    out = {"mode": "sort2", "metric": "Table 2 sorted by hash2, records/s", "unit": "records/s",
           "K": K, "table2_records": n2, "value": n2 / (ms / 1e3), "ms_per_sort": ms,
           "work_bytes": wb, "algorithmic_bytes": algo,
           "hbm": {"achieved_gbs": algo / (ms / 1e3) / 1e9, "peak_gbs": pk["hbm_gbs"],
                   "frac": algo / (ms / 1e3) / 1e9 / pk["hbm_gbs"]},
           "sorted_and_same_records": bool(ok), "steps": args.steps, "warmup": args.warmup,
           "data": "synthetic"}
    p.close()
    return out


def run_tiled(vx, args):
    """NEXT-4: a whole K plot built one window of whole logical buckets at a
    time in two window buffers (vx_plot_tiled), its tables copied to pinned
    host memory while the next window computes; wall-clock per plot (the
    call is synchronous).  Beside it, the whole plot in one device buffer set
    followed by the same copies (vx_plot_run, vx_sync, two device-to-host
    copies).  The tiled tables are checked on the host: Table-1 nonces are a
    permutation of 0..2^K-1 (sum and sum of squares), both counts equal the
    whole plot's."""
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    K, c = args.K, args.window_bits
    N = 1 << K
    key = plot_key(K)
    opts = plot_opts(vx, args)
    t1_out = not args.tiled_no_table1
    dev_bytes, h1b, h2b = vx.vx_plot_tiled_bytes(K, c, opts)
    whole_bytes = sum(vx.vx_plot_required_bytes(K, opts))
    h1 = torch.empty(h1b if t1_out else 0, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(h2b, dtype=torch.uint8, pin_memory=True)
    work = torch.empty(dev_bytes, dtype=torch.uint8, device="cuda")  # window buffers, allocated once
    stream = torch.cuda.current_stream()

    def tiled():
        rc, n1, n2 = vx.vx_plot_tiled(K, key, c, h1.data_ptr() if t1_out else 0, h1b if t1_out else 0,
                                      h2.data_ptr(), h2b, opts, stream, d_work=work.data_ptr(),
                                      work_bytes=work.numel())
        return n1, n2

    def wall(fn, steps):
        ts = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return sorted(ts)[len(ts) // 2] * 1e3, out

    for _ in range(args.warmup):
        tiled()
    ms_tiled, (n1, n2) = wall(tiled, args.steps)
    ok = n1 == N
    if t1_out:
        nonce = h1[: 12 * N].view(N, 12)[:, :4].contiguous().view(torch.int32).to(torch.int64)
        nonce &= 0xFFFFFFFF
        sq = ((N - 1) * N * (2 * N - 1) // 6) % (1 << 64)   # int64 sums wrap mod 2^64
        sq = sq - (1 << 64) if sq >= (1 << 63) else sq
        ok = ok and int(nonce.sum()) == N * (N - 1) // 2 and int((nonce * nonce).sum()) == sq
        del nonce
    out = {"mode": "tiled", "metric": "plot to host memory, nonces/s", "unit": "nonces/s",
           "K": K, "window_bits": c, "windows": 1 << c, "value": N / (ms_tiled / 1e3),
           "ms_per_plot": ms_tiled, "device_bytes": dev_bytes, "whole_plot_device_bytes": whole_bytes,
           "table1_copied": t1_out, "table1_records": n1, "table2_records": n2,
           "host_bytes_per_plot": (12 * n1 if t1_out else 0) + 16 * n2,
           "tables_check": bool(ok), "steps": args.steps, "warmup": args.warmup,
           "timing": "wall clock around the synchronous call, median of steps; window buffers "
                     "in one device buffer allocated before timing (as the whole plot's)",
           "data": "synthetic"}
    del work
    torch.cuda.empty_cache()
    if not args.tiled_no_whole:
        p = vx.Plot(K, key, opts)
        s2 = torch.cuda.Stream()

        def whole():
            p.run(stream)
            m2 = p.sync()
            torch.cuda.current_stream().wait_stream(stream)
            with torch.cuda.stream(s2):
                if t1_out:
                    h1[: 12 * N].copy_(p._t1[: 12 * N], non_blocking=True)
                h2[: 16 * m2].copy_(p._t2[: 16 * m2], non_blocking=True)
            s2.synchronize()
            return m2

        for _ in range(args.warmup):
            whole()
        ms_whole, m2 = wall(whole, args.steps)
        out.update({"whole_plot_ms_with_copy": ms_whole, "whole_table2_records": m2,
                    "tables_check": bool(ok and m2 == n2)})
        p.close()
    return out


def run_tiled_file(vx, args):
    """NEXT-4 + NEXT-1: a K plot built window by window with Table 2 streamed
    into a flat plot file (vx_plot_tiled_write), against the whole plot
    followed by vx_plot_write; wall clock per plot file, median of steps.
    The two files must be byte-identical."""
    import filecmp
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    K, c = args.K, args.window_bits
    key = plot_key(K)
    opts = plot_opts(vx, args)
    os.makedirs(args.tiled_file, exist_ok=True)
    fa = os.path.join(args.tiled_file, "tiled_k%d.plot" % K)
    fb = os.path.join(args.tiled_file, "whole_k%d.plot" % K)
    dev_bytes, _, _ = vx.vx_plot_tiled_bytes(K, c, opts)
    work = torch.empty(dev_bytes, dtype=torch.uint8, device="cuda")  # window buffers, allocated once
    stream = torch.cuda.current_stream()

    def tiled():
        _, n1, n2, sec = vx.vx_plot_tiled_write(K, key, c, fa, 0, 0, opts, stream,
                                                d_work=work.data_ptr(), work_bytes=work.numel())
        return n2

    p = vx.Plot(K, key, opts)

    def whole():
        p.run(stream)
        m2 = p.sync()
        vx.vx_plot_write(p.handle, fb)
        return m2

    # the two legs alternate step by step, so that both see the same state of
    # the host's page cache and disk
    for _ in range(args.warmup):
        tiled()
        whole()
    tt, tw, counts = [], [], {}
    for _ in range(args.steps):
        for name, fn, acc in (("tiled", tiled, tt), ("whole", whole, tw)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            counts[name] = fn()
            torch.cuda.synchronize()
            acc.append(time.perf_counter() - t0)
    n2, m2 = counts["tiled"], counts["whole"]
    ms_t = sorted(tt)[len(tt) // 2] * 1e3
    ms_w = sorted(tw)[len(tw) // 2] * 1e3
    same = n2 == m2 and filecmp.cmp(fa, fb, shallow=False)
    size = os.path.getsize(fa)
    p.close()
    for f in (fa, fb):
        os.remove(f)
    return {"mode": "tiled-file", "metric": "plot file written, nonces/s", "unit": "nonces/s",
            "K": K, "window_bits": c, "value": (1 << K) / (ms_t / 1e3), "ms_per_plot_file": ms_t,
            "whole_plot_ms_per_plot_file": ms_w, "file_bytes": size, "files_identical": bool(same),
            "steps_ms_tiled": [round(t * 1e3, 1) for t in tt], "steps_ms_whole": [round(t * 1e3, 1) for t in tw],
            "device_bytes": dev_bytes, "whole_plot_device_bytes": sum(vx.vx_plot_required_bytes(K, opts)),
            "steps": args.steps, "warmup": args.warmup,
            "timing": "wall clock around each synchronous call, median of steps", "data": "synthetic"}


def run_plotfile(vx, args):
    """One K plot file end to end, as the paper's totals count it (plot +
    write): a warm whole plot (vaultx.Plot), vx_plot_write and an fsync of
    the file; then the same file from vx_plot_tiled_write (window bits
    --window-bits, window buffers preallocated) and an fsync.  Skipped unless
    the directory has 2.5x the file free; the file is deleted after each
    leg."""
    import shutil
    import tempfile
    import torch
    from paper_2606_14007_gb300.inputs import plot_key
    K, c = args.K, args.window_bits
    base = args.tiled_file or tempfile.gettempdir()
    os.makedirs(base, exist_ok=True)
    st = os.statvfs(base)
    free = st.f_bavail * st.f_frsize
    need = 2.5 * 16 * (1 << K)
    out = {"mode": "plotfile", "metric": "plot file end to end, seconds", "unit": "s", "K": K,
           "higher_is_better": False, "dir_free_gb": round(free / 1e9, 1), "data": "synthetic"}
    if free < need:
        out["skipped"] = "less than %.0f GB free in %s" % (need / 1e9, base)
        return out
    d = tempfile.mkdtemp(prefix="vx_plotfile_", dir=base)
    path = os.path.join(d, "plot%d.bin" % K)

    def fsync(p_):
        fd = os.open(p_, os.O_RDONLY)
        os.fsync(fd)
        os.close(fd)

    try:
        p = vx.Plot(K, plot_key(K))
        p.run()
        p.sync()                          # warm-up, not timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.run()
        n2 = p.sync()
        t1 = time.perf_counter()
        vx.vx_plot_write(p.handle, path)
        t2 = time.perf_counter()
        fsync(path)
        t3 = time.perf_counter()
        size = os.path.getsize(path)
        p.close()
        del p
        torch.cuda.empty_cache()
        os.remove(path)
        out["whole"] = {"plot_s": t1 - t0, "write_s": t2 - t1, "fsync_s": t3 - t2, "total_s": t3 - t0,
                        "file_bytes": size, "write_GBps": size / (t2 - t1) / 1e9,
                        "device_bytes": sum(vx.vx_plot_required_bytes(K))}
        dev, _, _ = vx.vx_plot_tiled_bytes(K, c)
        work = torch.empty(dev, dtype=torch.uint8, device="cuda")
        t0 = time.perf_counter()
        _, _, m2, _ = vx.vx_plot_tiled_write(K, plot_key(K), c, path, d_work=work.data_ptr(),
                                             work_bytes=work.numel())
        t1 = time.perf_counter()
        fsync(path)
        t2 = time.perf_counter()
        out["tiled"] = {"window_bits": c, "device_bytes": dev, "write_call_s": t1 - t0,
                        "fsync_s": t2 - t1, "total_s": t2 - t0, "file_bytes": os.path.getsize(path),
                        "same_size": os.path.getsize(path) == size and m2 == n2}
        out["value"] = out["whole"]["total_s"]
    finally:
        shutil.rmtree(d, ignore_errors=True)
    return out


def run_mode(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_14007_gb300 import vaultx as vx
    from paper_2606_14007_gb300.inputs import batch_mix, plot_key
    if args.mode == "batch":
        mix = batch_mix(64, 20, 26, 2026, 1000)
        out = run_batch_compare(vx, mix, args.steps, args.warmup,
                                "aggregate nonces/s, 64 plots, K uniform in 20..26", "batch", args.autotune)
    elif args.mode == "large":
        mix = [(29, plot_key(3000 + i)) for i in range(4)] + [(27, plot_key(4000 + i)) for i in range(8)]
        out = run_batch_compare(vx, mix, args.steps, args.warmup,
                                "aggregate nonces/s, 4 x K=29 + 8 x K=27 sharing HBM", "large",
                                args.autotune)
    elif args.mode == "write":
        out = run_write(vx, args)
    elif args.mode == "sort2":
        out = run_sort2(vx, args)
    elif args.mode == "tiled":
        out = run_tiled_file(vx, args) if args.tiled_file else run_tiled(vx, args)
    elif args.mode == "plotfile":
        out = run_plotfile(vx, args)
    elif args.mode == "hashpeak":
        out = run_hashpeak(vx, args)
    elif args.mode == "sweep":
        out = run_sweep(vx, args)
    else:
        out = run_serve(vx, args)
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark: exact hierarchical (r,s) nucleus decomposition on one GB300.

Workload (one step): the (1,2), (2,3), (2,4) and (3,4) exact hierarchies of the R-MAT graph with
scale 18, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05), seed 2 (symmetrised, de-duplicated;
3.81M edges, 82.7M triangles): orientation, r-clique index (r = 1,2,3), s-clique counts, peel with
link-efficient and construct-tree for every pair.  value = s-cliques peeled per second of step
time (sum of n_s over the four pairs / step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (torchrun, one rank per GPU; the peel does not shard), value =
all ranks' s-cliques / max-over-ranks time.  --impl reference times the sequential CPU oracle on
a bounded sample of the same workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(r,s) hierarchy wall time & s-cliques peeled/sec on 1 GB300; HBM GB/s vs peak"
UNIT = "s-cliques/s"
PAIRS = [(1, 2), (2, 3), (2, 4), (3, 4)]
WORKLOAD = "RMAT scale 18 EF16 (0.57,0.19,0.19,0.05) seed 2; exact (1,2),(2,3),(2,4),(3,4) hierarchies"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=18, help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------------------------------------------
# reference arm: the sequential CPU oracle on a bounded sample
# -------------------------------------------------------------------------------------------------

def cpu_oracle_sample(scale: int = 15):
    """One bounded oracle run: (2,3) exact core numbers + definitional hierarchy of R-MAT scale
    `scale` EF16 seed 2, one host thread.  Returns (s-cliques, seconds)."""
    import oracle
    from paper_2306_08623_gb300 import graphgen as gg
    off, adj = gg.rmat(scale, 16, 2)
    t0 = time.perf_counter()
    res = oracle.nucleus(off, adj, 2, 3, hier="def")
    dt = time.perf_counter() - t0
    return res["n_s"], dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    scale = 15
    for _ in range(args.warmup):
        cpu_oracle_sample(scale)
    tot_s, tot_t = 0, 0.0
    for _ in range(args.steps):
        ns, dt = cpu_oracle_sample(scale)
        tot_s += ns
        tot_t += dt
    value = tot_s / tot_t
    sample = "RMAT scale %d EF16 seed 2, exact (2,3) core numbers + hierarchy, sequential oracle" % scale
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample, "l2": "inputs > L2 not needed (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------------------------------------
# our arm
# -------------------------------------------------------------------------------------------------

def algorithmic_peel_bytes(stats: dict, r: int, s: int) -> int:
    """Bytes the peel must move, from its own counters: every scanned adjacency entry (4 B), the
    round stamps of the other members of every re-listed s-clique (4 B each), every count
    decrement (4 B read + 4 B write), every triangle-table probe (one 16 B slot), every
    link-efficient call (uf + L entries, 8 B), every frontier entry (id + round + core, 12 B)."""
    from math import comb
    C = comb(s, r)
    return (4 * stats["scan_elements"] + 4 * (C - 1) * stats["s_cliques_listed"] + 8 * stats["decrements"]
            + 16 * stats["hash_probes"] + 8 * stats["link_calls"] + 12 * stats["frontier_total"])


def run_ours(args):
    import numpy as np
    import torch

    import paper_2306_08623_gb300.nucleus as nc
    from paper_2306_08623_gb300 import graphgen as gg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nc.lib()
    stream = torch.cuda.current_stream()

    off, adj = gg.rmat(args.scale, 16, 2)
    d_off = torch.from_numpy(off).to(dev)
    d_adj = torch.from_numpy(adj).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step(off_t, adj_t, timers=None, keep=None):
        o = nc.build_orientation(off_t, adj_t)
        ris = {r: nc.index_r_cliques(o, r) for r in sorted({p[0] for p in PAIRS})}
        n_s_tot = 0
        info = {}
        for r, s in PAIRS:
            ri = ris[r]
            cnt, n_s = nc.count_s_cliques(o, ri, s)
            if timers is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            pk = nc.peel_and_link(o, ri, s, cnt, stats=True)
            if timers is not None:
                b.record(stream)
                timers.setdefault((r, s), []).append((a, b))
            parent, label, nn = nc.construct_tree(pk["core"], pk["uf"], pk["L"])
            n_s_tot += n_s
            info[(r, s)] = {"n_r": ri.n_r, "n_s": n_s, "stats": pk["stats"], "n_nodes": nn}
            if keep is not None:
                keep.append((pk["core"], parent, label))
        return n_s_tot, info

    # warm-up
    for _ in range(args.warmup):
        n_s_tot, info = step(d_off, d_adj)
    torch.cuda.synchronize()

    # device-resident timed region
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = nc.kernel_launches()
    timers = {}
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1)  # L2 flush between steps (outside the step's events)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n_s_tot, info = step(d_off, d_adj, timers)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    launches = nc.kernel_launches() - launches0
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    value = world * n_s_tot * args.steps / (total_ms / 1000.0)

    # dominant kernel: the peel launch with the largest time
    peel_ms = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in timers.items()}
    dom = max(peel_ms, key=peel_ms.get)
    peak, peak_kind = measured_peaks()
    alg_bytes = algorithmic_peel_bytes(info[dom]["stats"], *dom)
    achieved = alg_bytes / (peel_ms[dom] / 1000.0) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "peel_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tt = json.load(f)
        if tt.get("kernel") == "k_peel<%d,%d,true>" % dom and tt.get("source_hash") == _source_hash():
            traffic = tt.get("dram_bytes_per_launch")

    # end to end through host buffers: H2D of the CSR from pinned memory, the path, D2H of
    # core / parent / label of every pair
    h_off = torch.from_numpy(off).pin_memory()
    h_adj = torch.from_numpy(adj).pin_memory()
    e2e_ms = []
    d2h = 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        off_t = h_off.to(dev, non_blocking=True)
        adj_t = h_adj.to(dev, non_blocking=True)
        keep = []
        step(off_t, adj_t, keep=keep)
        outs = []
        d2h = 0
        for core, parent, label in keep:
            for t in (core, parent, label):
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t, non_blocking=True)
                outs.append(h)
                d2h += t.numel() * t.element_size()
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_total = sum(e2e_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = world * n_s_tot * args.steps / (e2e_total / 1000.0)

    cpu = None
    if rank == 0 and world == 1:
        import oracle
        oracle.build()
        ns, dt = cpu_oracle_sample(15)
        cpu = {"value": ns / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "RMAT scale 15 EF16 seed 2, exact (2,3) core numbers + hierarchy, one host thread "
                         "(%d of %d cores), %.1f s" % (1, os.cpu_count() or 0, dt)}

    if rank == 0:
        per_pair = {"%d,%d" % k: {"n_r": v["n_r"], "n_s": v["n_s"], "nodes": v["n_nodes"],
                                  "rounds": v["stats"]["rounds"], "peel_ms": round(peel_ms[k], 3)}
                    for k, v in info.items()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "512 MiB buffer written between timed steps; step working set > L2",
                       "pairs": per_pair},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_peel<%d,%d,true> (%s peak)" % (dom[0], dom[1], peak_kind),
                         "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": peel_ms[dom]},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(off.nbytes + adj.nbytes),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_total / args.steps},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _source_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2306_08623_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2306_08623_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    args = parse()
    assert args.warmup >= 0 and args.steps >= 1
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

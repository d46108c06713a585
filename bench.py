#!/usr/bin/env python3
"""Benchmark of the batched protein database search on GB300.

Workload (default): 32 protein queries, lengths log-uniform in [64, 5000],
against a device-resident database of 500,000 targets with lognormal lengths
(median 300, sigma 0.7, cap 35,000), residues drawn from amino-acid
background frequencies; BLOSUM62, gap open 11 / extend 1, local alignment
with packed 16-bit lanes and exact int32 rerun on saturation; top-10 hits per
query with start coordinates and CIGAR.  A step is one `dsa_align` (score
pass + saturation rerun + top-k) plus one `dsa_traceback` of the hits.

Metric: GCUPS = (sum over pairs of m * n) / step time.  Printed as one JSON
line (rank 0).  `--impl reference` times the CPU oracle on a bounded sample
of the same workload instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS (bit-exact) batched protein database search"
# DRAM bytes per DP cell of k_inter_local16, from the ncu capture summarised in
# profiles/k_inter_local16_protein_8q_350k.md (416.4 GB read + written for
# 1.194 T cells); traffic grows with the cells (boundary rows per column and
# strip), so a launch's traffic is this figure times its cells.
INTER_DRAM_BYTES_PER_CELL = 416.40e9 / 1.194104e12
# the same figure for the global / semi-global form k_inter_glob16, from the
# capture summarised in profiles/k_inter_glob16_global_8q_350k.md (416.6 GB
# for the same 1.194 T cells)
GLOB_DRAM_BYTES_PER_CELL = 416.64e9 / 1.194104e12

# the workloads measured after the headline (each timed on its own)
SUB_WORKLOADS = ("reads_vs_windows", "long_pairs_global", "long_pairs_local",
                 "protein_search_global", "protein_search_semiglobal", "serving")

WORKLOAD = ("protein_search: 32 queries (log-uniform 64..5000) x 500,000 targets "
            "(lognormal median 300, sigma 0.7, cap 35,000), BLOSUM62 11/1, local, "
            "packed int16x2 + exact int32 rerun, top-10 + traceback")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--targets", type=int, default=500_000)
    ap.add_argument("--queries", type=int, default=32)
    ap.add_argument("--reads", type=int, default=1_000_000,
                    help="reads_vs_windows: number of reads (profiling runs use a smaller case)")
    ap.add_argument("--long-pairs", type=int, default=64,
                    help="long_pairs*: number of pairs (profiling runs use a smaller case)")
    ap.add_argument("--partition-residues", type=int, default=0,
                    help="protein_search: stream the host database through the device this many "
                         "residues at a time (partition + top-K reduce) instead of keeping it resident")
    ap.add_argument("--pssm", action="store_true",
                    help="protein_search: score against position-specific profiles (the queries' "
                         "BLOSUM62 rows perturbed by -2..+2) instead of the matrix; top-10 without "
                         "traceback (profile results carry scores and ends only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="approximate CPU time of the oracle sample")
    ap.add_argument("--requests", type=int, default=120,
                    help="serving: requests per measured load level")
    ap.add_argument("--no-workloads", action="store_true",
                    help="protein_search: skip the block of the other workloads")
    ap.add_argument("--workloads", default=",".join(SUB_WORKLOADS),
                    help="comma list of the other workloads measured after the headline")
    ap.add_argument("--sub-steps", type=int, default=3,
                    help="timed steps of each other workload")
    ap.add_argument("--sub-warmup", type=int, default=1,
                    help="untimed steps of each other workload (the headline's own warm-up "
                         "already ran the kernels)")
    ap.add_argument("--workload", default="protein_search",
                    choices=["protein_search", "protein_search_global", "protein_search_semiglobal",
                             "protein_vs_db", "reads_vs_windows", "long_pairs", "long_pairs_local",
                             "serving"],
                    help="the measured workload (default: the batched protein search)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, bus_id=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if bus_id:
            cmd += ["-i", bus_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------- distributed --

def dist_setup(args, backend="nccl"):
    """Rank layout from the launcher's environment; process group for N > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(world, x: float, op) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def all_max(world, x: float) -> float:
    """Slowest rank's time: the job's time."""
    import torch.distributed as dist
    return _reduce(world, x, dist.ReduceOp.MAX if world > 1 else None)


def all_sum(world, x: float) -> float:
    """Work of all ranks together."""
    import torch.distributed as dist
    return _reduce(world, x, dist.ReduceOp.SUM if world > 1 else None)


def aggregate(world, ms_local: float, cells_local: float):
    """(max ms over ranks, total cells, whole-job GCUPS) for weak scaling."""
    ms = all_max(world, ms_local)
    cells = all_sum(world, cells_local)
    return ms, cells, cells / (ms / 1e3) / 1e9


# ---------------------------------------------------------------- workload --

def make_workload(args, rank=0):
    from paper_1701_01575_gb300 import workloads as W
    if args.workload == "protein_vs_db":
        return W.protein_vs_db(seed=W.SEED_BASE + 0 + 1000 * rank)
    if args.workload == "reads_vs_windows":
        return W.reads_vs_windows(seed=W.SEED_BASE + 2 + 1000 * rank, n_reads=args.reads)
    if args.workload in ("long_pairs", "long_pairs_local"):
        mode = W.MODE_LOCAL if args.workload == "long_pairs_local" else W.MODE_GLOBAL
        return W.long_pairs(seed=W.SEED_BASE + 3 + 1000 * rank, mode=mode, n_pairs=args.long_pairs)
    # protein search: rank r holds shard r of one database (targets
    # r * targets .. (r + 1) * targets - 1 in global numbering; shard 0 is the
    # one-GPU database) and every rank the same queries
    wl = W.protein_search(seed=W.SEED_BASE + 1 + 1000 * rank, n_queries=args.queries,
                          n_targets=args.targets)
    if rank:
        wl.queries = W.protein_search(seed=W.SEED_BASE + 1, n_queries=args.queries,
                                      n_targets=1).queries
    wl.meta["target_base"] = rank * args.targets
    if args.workload in ("protein_search_global", "protein_search_semiglobal"):
        wl.mode = W.MODE_GLOBAL if args.workload.endswith("_global") else W.MODE_SEMIGLOBAL
    return wl


def gather_merge(world, rank, hits, cigar, n_queries, k, target_base):
    """Partition top-K reduce across ranks (Sec. II.B.2): every rank's top-K
    hits (shard-local target ids) and CIGAR words go to rank 0, which merges
    them under (score desc, global target id asc) with dsa_merge_topk.
    Returns (hits, cigar) with global target ids on rank 0, None elsewhere."""
    from paper_1701_01575_gb300 import dsa
    mine = (hits.tobytes(), cigar.tobytes(), int(target_base))
    if world > 1:
        import torch.distributed as dist
        lists = [None] * world
        dist.all_gather_object(lists, mine)
    else:
        lists = [mine]
    if rank != 0:
        return None
    parts = [(np.frombuffer(h, dtype=dsa.HIT_DTYPE), np.frombuffer(c, dtype=np.uint32))
             for h, c, _ in lists]
    return dsa.merge_topk(parts, [b for _, _, b in lists], n_queries, k)


WORKLOAD_TEXT = {
    "protein_search_global": WORKLOAD.replace(", local,", ", global,"),
    "protein_search_semiglobal": WORKLOAD.replace(", local,", ", semi-global (all four ends free),"),
    "protein_vs_db": "protein_vs_db: 1 query of 128 x 2,000 targets U{50..500}, BLOSUM62 11/1, local",
    "reads_vs_windows": ("reads_vs_windows: 1,000,000 reads (150/250 bp, 1% subs, 0.1% indels) vs "
                         "500 bp windows of a 10 Mb genome, +1/-4, 6/1, semi-global (target ends "
                         "free), score + traceback of every read"),
    "long_pairs": ("long_pairs: 64 DNA pairs log-uniform 1e4..1e5 (5% subs, 1% indels), +2/-3, "
                   "5/2, global, score + traceback"),
    "long_pairs_local": ("long_pairs: 64 DNA pairs log-uniform 1e4..1e5 (5% subs, 1% indels), "
                         "+2/-3, 5/2, local, score + traceback"),
}


def cpu_sample(wl, seconds, rate_guess=0.25e9):
    """A seeded sample of targets (all queries against each) sized to ~`seconds` of CPU."""
    cores = os.cpu_count() or 1
    budget = seconds * rate_guess * cores
    qsum = int(wl.queries.lengths.sum())
    mean_n = float(wl.db.lengths.mean())
    k = max(8, min(wl.db.n, int(budget / (qsum * mean_n))))
    rng = np.random.default_rng(20260101)
    return np.sort(rng.choice(wl.db.n, size=k, replace=False)), cores


def run_oracle_sample(wl, targets, cores):
    import oracle
    t0 = time.perf_counter()
    sc, qe, te = oracle.score_all_vs_all(wl.queries, wl.db, wl.matrix, wl.gap_open, wl.gap_extend,
                                         oracle.LOCAL, 15, targets=targets, threads=cores)
    dt = time.perf_counter() - t0
    cells = int(wl.queries.lengths.sum()) * int(wl.db.lengths[targets].sum())
    return (sc, qe, te), cells, dt


# ------------------------------------------------------------------ ours --

def bench_ours(args):
    import torch
    from paper_1701_01575_gb300 import build, dsa

    world, rank, local = dist_setup(args)
    build.build()
    torch.cuda.set_device(local)
    # an explicit stream: the library orders all its work on it and the CUDA
    # events below are recorded on it
    stream = torch.cuda.Stream(local)
    torch.cuda.set_stream(stream)
    wl = make_workload(args, rank)
    ctx = dsa.Context(local, stream=stream)
    A = wl.alphabet_size
    db = ctx.load_set(wl.db, A)
    qs = ctx.load_set(wl.queries, A)
    S, o, e = wl.matrix, wl.gap_open, wl.gap_extend
    cells_per_step = wl.cells()
    flags = dsa.TIMING | dsa.RESULTS_ON_DEVICE

    pairs_dev = None
    if wl.pairs is not None:
        pairs_dev = torch.as_tensor(wl.pairs.view(np.uint8), device="cuda")

    pssm = None
    if args.pssm:
        from paper_1701_01575_gb300 import workloads as W
        prng = np.random.default_rng(W.SEED_BASE + 77)
        pssm = np.clip(S[wl.queries.codes].astype(np.int16) + prng.integers(-2, 3, (len(wl.queries.codes), A)),
                       -128, 127).astype(np.int8)

    def step():
        if pssm is not None:
            return ctx.align_pssm(db, qs, pssm, o, e, mode=wl.mode, free_ends=wl.free_ends,
                                  top_k=wl.top_k, flags=flags)
        if args.partition_residues:
            # every step loads each partition from host memory, searches and
            # traces it, and merges the per-partition top-K lists
            return ctx.search_partitioned(wl.db.codes, wl.db.offsets, A, qs, S, o, e, wl.top_k,
                                          args.partition_residues, mode=wl.mode,
                                          free_ends=wl.free_ends)
        r = ctx.align(db, qs, S, o, e, mode=wl.mode, free_ends=wl.free_ends, pairs=pairs_dev,
                      top_k=wl.top_k, flags=flags)
        ctx.traceback(r)
        return r

    for _ in range(args.warmup):
        step().free()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)
    launches0 = ctx.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(bus)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    launches = ctx.kernel_launches() - launches0
    ms_local = ev0.elapsed_time(ev1)
    phase = {k: [] for k in dsa.PHASES}
    reruns = 0
    pcells = results[0].phase_cells()
    for r in results:
        t = r.timing()
        for k, v in t.items():
            if v >= 0:
                phase[k].append(v)
        reruns += r.stats()[1]
    last = results[-1]
    top_hits = last.hits()
    top_cigar = last.cigar()
    for r in results:
        r.free()
    merged = None
    if args.workload.startswith("protein_search") and wl.top_k and not args.pssm:
        # the shards' top-K lists, merged on rank 0 (outside the timed region)
        t_m = time.perf_counter()
        got = gather_merge(world, rank, top_hits, top_cigar, wl.queries.n, wl.top_k,
                           wl.meta["target_base"])
        if got is not None:
            mh, mc = got
            merged = {"ranks": world, "hits": int(len(mh)), "cigar_words": int(len(mc)),
                      "top_q0": [(int(h["target_id"]), int(h["score"])) for h in mh[:3]],
                      "host_ms": round((time.perf_counter() - t_m) * 1e3, 1)}
    ms, total_cells, value = aggregate(world, ms_local, float(cells_per_step * args.steps))

    wtext = WORKLOAD if args.workload == "protein_search" else WORKLOAD_TEXT[args.workload]
    if args.workload.startswith("protein_search"):
        wtext = wtext.replace("32 queries", f"{wl.queries.n} queries").replace(
            "500,000 targets", f"{wl.db.n:,} targets")
    if args.workload == "reads_vs_windows":
        wtext = wtext.replace("1,000,000 reads", f"{args.reads:,} reads")
    if args.workload.startswith("long_pairs"):
        wtext = wtext.replace("64 DNA pairs", f"{args.long_pairs} DNA pairs")
    if args.pssm:
        wtext = wtext.replace("BLOSUM62 11/1", "position-specific profiles (BLOSUM62 rows of each "
                              "query residue + uniform -2..2), 11/1").replace(" + traceback", "")
    if args.partition_residues:
        wtext += (f"; database streamed from host memory in partitions of {args.partition_residues:,} "
                  "residues, per-partition top-K merged")
    out = {"metric": METRIC if args.workload == "protein_search" else
           f"GCUPS (bit-exact) {args.workload}", "value": round(value, 2), "unit": "GCUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i16x2+i32",
           "data": "synthetic",
           "config": {"workload": wtext, "queries": wl.queries.n, "targets": wl.db.n,
                      "cells_per_step": cells_per_step,
                      "parallelism": (f"database shards x{world}, per-shard top-K merged on rank 0"
                                      if args.workload.startswith("protein_search")
                                      else f"replicas x{world}"),
                      "l2": "inputs larger than L2" if wl.db.codes.nbytes + wl.queries.codes.nbytes > (129 << 20)
                      else "inputs smaller than L2 (small workload)"},
           "clocks": clk, "gpu_launches": int(launches)}

    # roofline of the dominant kernel (packed inter-sequence kernel)
    inter_ms = statistics.mean(phase["inter16"]) if phase["inter16"] else None
    if not args.workload.startswith("protein_search"):
        inter_ms = None
    kname = "k_inter_local16" if args.workload == "protein_search" else "k_inter_glob16"
    rate = ctx.probe_issue_rate(0)      # DPX s16x2 add-max, warp-instr / SM / clk
    rate_add = ctx.probe_issue_rate(3)  # 32-bit integer add, warp-instr / SM / clk
    sm_mhz = clk.get("sm_mhz") or (props.clock_rate / 1e3 if hasattr(props, "clock_rate") else None)
    if inter_ms and sm_mhz:
        achieved = pcells["inter16"] / (inter_ms / 1e3) / 1e9
        # 6 algorithmic ops per cell (H-o, E, F, max with diagonal, max with F/0, running
        # best), each at the measured rate of the form the kernel uses: five maxima as
        # DPX s16x2 instructions, H - o as one 32-bit add over both offset-binary halves;
        # every instruction covers 2 cells of 32 lanes
        peak = (props.multi_processor_count * sm_mhz * 1e6 * 32 * 2 / (5 / rate + 1 / rate_add)
                / 1e9)
        per_cell = INTER_DRAM_BYTES_PER_CELL if kname == "k_inter_local16" else GLOB_DRAM_BYTES_PER_CELL
        out["roofline"] = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1),
                           "unit": "GCUPS", "frac": round(achieved / peak, 4),
                           "traffic": round(per_cell * pcells["inter16"]) if per_cell else None,
                           "traffic_basis": "ncu dram__bytes_read+write of an 8-query x 350k "
                                            "capture, scaled by cells to this launch",
                           "kernel": kname, "kernel_ms": round(inter_ms, 3),
                           "peak_basis": f"{props.multi_processor_count} SMs x {sm_mhz:.0f} MHz x "
                                         "32 lanes x 2 cells / (5 DPX ops / "
                                         f"{rate:.3f} + 1 add / {rate_add:.3f} warp-instr/SM/clk, "
                                         "both measured)"}
    out["phases_ms"] = {k: round(statistics.mean(v), 3) for k, v in phase.items() if v}
    out["phase_gcups"] = {k: round(pcells[k] / (statistics.mean(v) / 1e3) / 1e9, 1)
                          for k, v in phase.items() if v and pcells.get(k)}
    out["saturation_reruns_per_step"] = reruns / args.steps

    if rank == 0 and not args.no_plain and args.workload == "protein_search":
        # plain per-query form: one unbatched int32 launch per query, DB in input order
        from paper_1701_01575_gb300 import workloads as W
        order = np.argsort(wl.queries.lengths)
        pick = order[[len(order) // 8, 3 * len(order) // 8, 5 * len(order) // 8, 7 * len(order) // 8]]
        sub = wl.queries.subset(pick)
        qsub = ctx.load_set(sub, A)
        r = ctx.align(db, qsub, S, o, e, flags=dsa.PLAIN_FORM | dsa.TIMING | dsa.RESULTS_ON_DEVICE)
        ctx.sync()
        r.free()
        t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        r = ctx.align(db, qsub, S, o, e, flags=dsa.PLAIN_FORM | dsa.RESULTS_ON_DEVICE)
        t1.record(stream)
        torch.cuda.synchronize()
        r.free()
        pms = t0.elapsed_time(t1)
        pcells = int(sub.lengths.sum()) * int(wl.db.lengths.sum())
        plain = pcells / (pms / 1e3) / 1e9
        out["plain_form"] = {"value": round(plain, 2), "unit": "GCUPS",
                             "sample": "4 of the 32 queries (length quantiles 1/8..7/8) x all "
                                       "targets, one int32 launch per query"}
        out["batched_over_plain"] = round(value / world / plain, 2)
        qsub.free()

    if rank == 0 and not args.no_e2e and args.workload == "protein_search":
        # end to end through the public API with host buffers: queries H2D, hits + CIGAR D2H
        e2e_steps = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(e2e_steps):
            r = ctx.align_batch(db, wl.queries.codes, wl.queries.offsets, S, o, e, top_k=wl.top_k)
            ctx.traceback(r)
            hits = r.hits()
            cig = r.cigar()
            h2d += wl.queries.codes.nbytes + wl.queries.offsets.nbytes
            d2h += hits.nbytes + cig.nbytes
            r.free()
        dt = time.perf_counter() - t0
        out["e2e"] = {"value": round(cells_per_step * e2e_steps / dt / 1e9, 2), "unit": "GCUPS",
                      "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
                      "steps": e2e_steps}

    if rank == 0 and not args.no_cpu_baseline and args.workload == "protein_search":
        targets, cores = cpu_sample(wl, args.cpu_seconds)
        (osc, oqe, ote), ccells, cdt = run_oracle_sample(wl, targets, cores)
        out["cpu_baseline"] = {"value": round(ccells / cdt / 1e9, 4), "unit": "GCUPS", "cores": cores,
                               "kind": "oracle",
                               "sample": f"all {wl.queries.n} queries x {len(targets)} seeded random "
                                         f"targets ({ccells:.3g} cells, {cdt:.1f} s)"}
        # the same sample, checked against the GPU's dense all-pairs result (packed path)
        r = ctx.align(db, qs, S, o, e, flags=dsa.RESULTS_ON_DEVICE)
        dh = r.device_hits().view(-1, dsa.HIT_DTYPE.itemsize)
        import torch as _t
        idx = (_t.arange(wl.queries.n, device="cuda")[:, None] * wl.db.n
               + _t.as_tensor(targets, device="cuda")[None, :]).reshape(-1)
        sel = dh.index_select(0, idx).cpu().numpy().view(dsa.HIT_DTYPE).reshape(wl.queries.n, -1)
        r.free()
        mism = int((sel["score"] != osc).sum() + (sel["q_end"] != oqe).sum() + (sel["t_end"] != ote).sum())
        out["cpu_baseline"]["parity_mismatches"] = mism
        out["top_hits_q0"] = [(int(h["target_id"]), int(h["score"])) for h in top_hits[:3]]

    if rank == 0 and not args.no_workloads and args.workload == "protein_search" and \
            not args.pssm and not args.partition_residues:
        # the other workloads, each timed on its own after the headline
        out["workloads"] = {}
        for name in [x for x in args.workloads.split(",") if x]:
            if name == "serving":
                out["workloads"][name] = serving_block(args, bus, protein_db=wl.db)
            else:
                out["workloads"][name] = sub_workload(name, args, ctx, stream, bus, (wl, db, qs))

    if merged is not None:
        out["merge"] = merged
    if rank == 0:
        print(json.dumps(out), flush=True)
    qs.free(); db.free(); ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------- other workloads --

def timed_steps(ctx, stream, step, steps, warmup, bus):
    """`warmup` untimed steps, then `steps` steps between CUDA events recorded on
    the library's stream, with the clocks sampled meanwhile.  Returns (ms,
    results, clocks, kernel launches)."""
    import torch
    for _ in range(warmup):
        step().free()
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches()
    clocks = ClockSampler(bus)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [step() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return ev0.elapsed_time(ev1), results, clk, ctx.kernel_launches() - launches0


def phase_summary(results):
    """Mean device milliseconds and GCUPS of each phase the results recorded."""
    from paper_1701_01575_gb300 import dsa
    phase = {k: [] for k in dsa.PHASES}
    for r in results:
        for k, v in r.timing().items():
            if v >= 0:
                phase[k].append(v)
    pcells = results[0].phase_cells()
    ms = {k: round(statistics.mean(v), 3) for k, v in phase.items() if v}
    gc = {k: round(pcells[k] / (statistics.mean(v) / 1e3) / 1e9, 1)
          for k, v in phase.items() if v and pcells.get(k)}
    return ms, gc


def _pairs_parity(wl, h, cig, pick, trace_every):
    """Oracle scores and ends of the sampled pairs, begins and CIGARs of every
    `trace_every`-th of them: the number of fields that differ."""
    import oracle
    p = wl.pairs[pick]
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix,
                                    wl.gap_open, wl.gap_extend, wl.mode, wl.free_ends,
                                    pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    hs = h[pick]
    bad = int((hs["score"] != sc).sum() + (hs["q_end"] != qe).sum() + (hs["t_end"] != te).sum())
    for k in range(0, len(pick), trace_every):
        x = hs[k]
        if wl.mode == 0 and x["score"] == 0:
            continue
        t0 = int(wl.db.offsets[int(x["target_id"])]) + int(x["t_offset"])
        t = wl.db.codes[t0:t0 + int(p["t_len"][k])]
        qb, tb, c = oracle.traceback(wl.queries.seq(int(x["query_id"])), t, wl.matrix, wl.gap_open,
                                     wl.gap_extend, wl.mode, wl.free_ends, int(x["q_end"]),
                                     int(x["t_end"]))
        got = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        bad += int((int(x["q_begin"]), int(x["t_begin"])) != (qb, tb)) + int(got.tolist() != c.tolist())
    return bad


def _hits_parity(wl, h, cig, max_trace_cells=30_000_000):
    """Oracle score and ends of every reported all-vs-all hit; begins and CIGAR
    of those whose rectangle has at most `max_trace_cells` cells."""
    import oracle
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, h["query_id"], h["target_id"], wl.matrix,
                                    wl.gap_open, wl.gap_extend, wl.mode, wl.free_ends)
    bad = int((h["score"] != sc).sum() + (h["q_end"] != qe).sum() + (h["t_end"] != te).sum())
    traced = 0
    for x in h:
        if (int(x["q_end"]) + 1) * (int(x["t_end"]) + 1) > max_trace_cells:
            continue
        qb, tb, c = oracle.traceback(wl.queries.seq(int(x["query_id"])),
                                     wl.db.seq(int(x["target_id"])), wl.matrix, wl.gap_open,
                                     wl.gap_extend, wl.mode, wl.free_ends, int(x["q_end"]),
                                     int(x["t_end"]))
        got = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        bad += int((int(x["q_begin"]), int(x["t_begin"])) != (qb, tb)) + int(got.tolist() != c.tolist())
        traced += 1
    return bad, traced


# score-pass kernel of each other workload: (phase, kernel, packed int16x2?)
# phase, score-pass kernel, packed (2 cells per instruction), and the kernel's
# ops per register and row: maxima (DPX) and plain adds
SUB_KERNELS = {"reads_vs_windows": ("inter16", "k_pairs16", True, 5, 1),
               "long_pairs_global": ("intra16", "k_long_score16", True, 5, 1),
               "long_pairs_local": ("intra16", "k_long_score16", True, 5.5, 0),
               "protein_search_global": ("inter16", "k_inter_glob16", True, 5, 1),
               "protein_search_semiglobal": ("inter16", "k_inter_glob16", True, 5, 1)}


def sub_roofline(name, ctx, clk, phase_gcups):
    """The score-pass kernel against the ALU-pipe roofline of its form: the
    maxima at the measured DPX rate (s16x2 for the packed kernels, 2 cells per
    instruction; s32 for the int32 kernel, 1) and the adds at the measured
    integer-add rate, 32 lanes per instruction.  Global forms take five
    maxima and one add (H - o) per register and row; the local long-pair form
    folds the floor into a sixth maximum in place of the add and keeps a
    three-way running maximum every two rows (5.5 maxima)."""
    import torch
    if name not in SUB_KERNELS or not clk.get("sm_mhz"):
        return None
    phase, kernel, packed, n_max, n_add = SUB_KERNELS[name]
    if phase not in phase_gcups:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    rate_max = ctx.probe_issue_rate(0 if packed else 6)
    rate_add = ctx.probe_issue_rate(3)
    cells = 2 if packed else 1
    peak = sms * clk["sm_mhz"] * 1e6 * 32 * cells / (n_max / rate_max + n_add / rate_add) / 1e9
    achieved = phase_gcups[phase]
    add_txt = f" + {n_add} add / {rate_add:.3f}" if n_add else ""
    return {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 1),
            "peak": round(peak, 1), "unit": "GCUPS", "frac": round(achieved / peak, 4),
            "peak_basis": f"{sms} SMs x {clk['sm_mhz']:.0f} MHz x 32 lanes x {cells} cell(s) / "
                          f"({n_max} {'DPX s16x2' if packed else 'DPX s32'} ops / {rate_max:.3f}"
                          f"{add_txt} warp-instr/SM/clk, measured)"}


def sub_workload(name, args, ctx, stream, bus, main):
    """One of the other workloads, measured like the headline: its own warm-up,
    timed steps (align + traceback of every hit) on the library's stream, clock
    record and an oracle-sample parity count.  `main` = (workload, db, queries)
    of the headline, reused by the global and semi-global searches."""
    import torch
    from paper_1701_01575_gb300 import dsa
    from paper_1701_01575_gb300 import workloads as W
    flags = dsa.TIMING | dsa.RESULTS_ON_DEVICE
    t_gen = time.perf_counter()
    own = []
    if name == "reads_vs_windows":
        wl = W.reads_vs_windows(seed=W.SEED_BASE + 2, n_reads=args.reads)
        text = WORKLOAD_TEXT["reads_vs_windows"].replace("1,000,000 reads", f"{args.reads:,} reads")
    elif name in ("long_pairs_global", "long_pairs_local"):
        mode = W.MODE_LOCAL if name == "long_pairs_local" else W.MODE_GLOBAL
        wl = W.long_pairs(seed=W.SEED_BASE + 3, mode=mode, n_pairs=args.long_pairs)
        text = WORKLOAD_TEXT["long_pairs" if mode == W.MODE_GLOBAL else "long_pairs_local"]
        text = text.replace("64 DNA pairs", f"{args.long_pairs} DNA pairs")
    else:
        mwl, db, qs = main
        mode = W.MODE_GLOBAL if name == "protein_search_global" else W.MODE_SEMIGLOBAL
        wl = W.Workload(name, mwl.queries, mwl.db, mwl.matrix, mwl.gap_open, mwl.gap_extend, mode,
                        free_ends=15, top_k=mwl.top_k, meta=mwl.meta)
        text = WORKLOAD.replace(", local,", ", global," if mode == W.MODE_GLOBAL else
                                ", semi-global (all four ends free),")
    gen_s = time.perf_counter() - t_gen
    if wl.pairs is not None:
        db = ctx.load_set(wl.db, wl.alphabet_size)
        qs = ctx.load_set(wl.queries, wl.alphabet_size)
        own = [db, qs]
        pairs = torch.as_tensor(wl.pairs.view(np.uint8), device="cuda")
    else:
        pairs = None

    def step():
        r = ctx.align(db, qs, wl.matrix, wl.gap_open, wl.gap_extend, mode=wl.mode,
                      free_ends=wl.free_ends, pairs=pairs, top_k=wl.top_k, flags=flags)
        ctx.traceback(r)
        return r

    ms, results, clk, launches = timed_steps(ctx, stream, step, args.sub_steps, args.sub_warmup, bus)
    phases_ms, phase_gcups = phase_summary(results)
    cells = wl.cells()
    last = results[-1]
    h, cig = last.hits(), last.cigar()
    for r in results:
        r.free()
    t_par = time.perf_counter()
    if wl.pairs is not None:
        if name == "reads_vs_windows":
            pick = np.sort(np.random.default_rng(11).choice(len(wl.pairs), 2000, replace=False))
            sample = "2,000 seeded random reads (score, ends), begins + CIGAR of every 10th"
            bad = _pairs_parity(wl, h, cig, pick, 10)
        else:
            sizes = wl.queries.lengths * wl.pairs["t_len"].astype(np.int64)
            pick = np.sort(np.argsort(sizes)[:3])
            sample = "the 3 smallest pairs (score, ends, begins, CIGAR)"
            bad = _pairs_parity(wl, h, cig, pick, 1)
    else:
        bad, traced = _hits_parity(wl, h, cig)
        sample = (f"all {len(h)} reported hits (score, ends); begins + CIGAR of the {traced} "
                  "hits of at most 3e7 cells")
    out = {"workload": text, "metric": "GCUPS (bit-exact)", "value": round(cells * args.sub_steps
                                                                          / (ms / 1e3) / 1e9, 2),
           "unit": "GCUPS", "steps": args.sub_steps, "warmup": args.sub_warmup,
           "ms_per_step": round(ms / args.sub_steps, 3), "cells_per_step": int(cells),
           "phases_ms": phases_ms, "phase_gcups": phase_gcups, "gpu_launches": int(launches),
           "clocks": clk, "parity": {"sample": sample, "mismatches": bad},
           "host_s": {"generate": round(gen_s, 1), "oracle": round(time.perf_counter() - t_par, 1)}}
    roof = sub_roofline(name, ctx, clk, phase_gcups)
    if roof:
        out["roofline"] = roof
    for x in own:
        x.free()
    return out


# ---------------------------------------------------------------- serving --

SERVING_TEXT = ("serving: Poisson arrivals, 70% protein queries (log-uniform 50..2000) vs 500,000 "
                "targets top-10 + traceback, 30% DNA read batches (log-uniform 1e3..1e5 reads of "
                "150 bp vs 500 bp windows of a 10 Mb genome) with traceback; 2 slots")


def serving_block(args, bus=None, protein_db=None):
    """Serving loop: sustained capacity C (a burst of requests), then Poisson
    loads at 0.5 C and 0.8 C; latency from arrival to result ready, queueing
    included.  `protein_db`: the 500,000-target database (host arrays) if it
    exists already.  Returns the capacity and the per-load figures."""
    from paper_1701_01575_gb300 import dsa
    from paper_1701_01575_gb300 import workloads as W
    t_gen = time.perf_counter()
    rng = np.random.default_rng(W.SEED_BASE + 4)
    if protein_db is None:
        protein_db = W.protein_search(seed=W.SEED_BASE + 1, n_queries=1, n_targets=args.targets).db
    genome = rng.integers(0, 4, 10_000_000).astype(np.uint8)
    gdb = W.SeqSet(genome, np.array([0, len(genome)], dtype=np.uint64))
    ctx = dsa.Context(0)
    d_p = ctx.load_set(protein_db, 24)
    d_g = ctx.load_set(gdb, 4)
    db_res = int(protein_db.codes.nbytes)
    S_p, S_d = W.blosum62(), W.dna_matrix(1, -4)

    def cells(r):
        if r.kind == "protein":
            return int(r.queries.lengths.sum()) * db_res
        return int(r.queries.lengths.sum()) * 500

    def submit(srv, r):
        if r.kind == "protein":
            return srv.submit(d_p, r.queries.codes, r.queries.offsets, S_p, 11, 1, top_k=10,
                              traceback=True)
        return srv.submit(d_g, r.queries.codes, r.queries.offsets, S_d, 6, 1, mode=dsa.SEMIGLOBAL,
                          free_ends=W.FREE_T_BEGIN | W.FREE_T_END, pairs=r.pairs, traceback=True)

    def run(reqs, rate):
        srv = dsa.Server(0, n_slots=2)
        t0 = srv.now()
        tickets = []
        for r in reqs:
            if rate:
                delay = t0 + r.arrival - srv.now()
                if delay > 0:
                    time.sleep(delay)
            tickets.append(submit(srv, r))
        srv.drain()
        lat, fin, arr, batch = [], [], [], []
        for t in tickets:
            res, tm = srv.poll(t)
            assert res is not None, tm
            lat.append(tm["finish"] - tm["arrive"])
            fin.append(tm["finish"])
            arr.append(tm["arrive"])
            batch.append(tm["batch_requests"])
            res.free()
        srv.close()
        span = max(fin) - min(arr)
        total = sum(cells(r) for r in reqs)
        lat = np.array(lat)
        return {"requests": len(reqs), "span_s": round(span, 3),
                "gcups": round(total / span / 1e9, 1),
                "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
                "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
                "max_ms": round(float(lat.max()) * 1e3, 2),
                "mean_batch": round(float(np.mean(batch)), 2)}

    n = args.requests
    warm = W.serving_stream(seed=W.SEED_BASE + 40, n_requests=8, rate=1e9, genome=genome)
    burst = W.serving_stream(seed=W.SEED_BASE + 41, n_requests=n, rate=1e9, genome=genome)
    # the load streams' arrival times are scaled to the measured capacity below
    load_reqs = {frac: W.serving_stream(seed=W.SEED_BASE + 42 + int(frac * 10), n_requests=n,
                                        rate=1.0, genome=genome) for frac in (0.5, 0.8)}
    gen_s = time.perf_counter() - t_gen
    run(warm, 0)
    clocks = ClockSampler(bus)
    cap = run(burst, 0)
    C = cap["requests"] / cap["span_s"]
    loads = {}
    for frac, reqs in load_reqs.items():
        for r in reqs:
            r.arrival /= frac * C   # Poisson at rate 1 -> rate frac * C
        loads[f"{frac}C"] = dict(run(reqs, frac * C), rate_per_s=round(frac * C, 2))
    clk = clocks.stop()
    d_p.free(); d_g.free(); ctx.close()
    return {"workload": SERVING_TEXT, "requests_per_level": n,
            "capacity": dict(cap, requests_per_s=round(C, 2)), "loads": loads, "clocks": clk,
            "parity": {"sample": "results identical alone and in the mix: tests/test_gpu_serving.py",
                       "mismatches": None},
            "host_s": {"generate": round(gen_s, 1)}}


def bench_serving(args):
    """Serving loop alone: capacity, then Poisson loads at 0.5 and 0.8 of it."""
    from paper_1701_01575_gb300 import build
    build.build()
    blk = serving_block(args)
    loads = blk["loads"]
    out = {"metric": "serving: p50/p99 request latency and GCUPS at 0.8 of capacity",
           "value": loads["0.8C"]["p99_ms"], "unit": "ms (p99)", "n_gpus": 1,
           "higher_is_better": False, "data": "synthetic", "dtype": "i16x2+i32",
           "config": {"workload": SERVING_TEXT, "requests_per_level": blk["requests_per_level"]},
           "capacity": blk["capacity"], "loads": loads, "clocks": blk["clocks"]}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------- reference --

def bench_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args, 0)
    per_step = max(1.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    targets, cores = cpu_sample(wl, per_step)
    for _ in range(args.warmup):
        run_oracle_sample(wl, targets[: max(8, len(targets) // 8)], cores)
    total_cells, total_t = 0, 0.0
    for _ in range(args.steps):
        _, cells, dt = run_oracle_sample(wl, targets, cores)
        total_cells += cells
        total_t += dt
    value = total_cells / total_t / 1e9
    out = {"metric": METRIC, "value": round(value, 4), "unit": "GCUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(total_t / args.steps * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "queries": args.queries, "targets": args.targets},
           "cpu_baseline": {"value": round(value, 4), "unit": "GCUPS", "cores": cores,
                            "kind": "oracle",
                            "sample": f"per step all {wl.queries.n} queries x {len(targets)} "
                                      "seeded random targets"},
           "e2e": {"value": round(value, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        bench_reference(a)
    elif a.workload == "serving":
        bench_serving(a)
    else:
        bench_ours(a)
